/*
 * libofdft: finite-temperature orbital-free DFT on one GB300 GPU.
 *
 * C ABI for the data-parallel hot path of finite-T OF-DFT molecular dynamics
 * (arXiv:1406.0835, Karasiev, Sjostrom, Trickey): the non-interacting free
 * energy (ftTF, SGA, ftGGA/VT84F, KST2-family) plus Hartree, local
 * pseudopotential and LDA XC terms and their functional derivative on a
 * periodic 3D grid, its minimisation over phi = sqrt(n) under the
 * electron-number constraint, Hellmann-Feynman and Ewald forces, the pressure
 * and the MD step.  The calls mirror the paper's interface
 *   profess(nat, tau, force, pressure, etot, einternel)   (Sec. V C)
 * split into setup / energy / minimise / forces / MD step.
 *
 * Conventions (all calls):
 *  - Hartree atomic units (Sec. I units note); temperatures in kelvin (the
 *    TEMP keyword of Sec. V B).  Positions are Cartesian bohr.
 *  - Grid fields are C-order [ix][iy][iz] with iz fastest, point
 *    (ix,iy,iz) at (ix Lx/nx, iy Ly/ny, iz Lz/nz).
 *  - Every host pointer belongs to the caller and is only read or written
 *    during the call; the library copies what it keeps.  The library owns all
 *    device memory of a context until ofdft_destroy.
 *  - Calls on one context are not thread-safe; distinct contexts are.
 *  - Every call returns an ofdft_status.  On error, outputs are left
 *    untouched (except ofdft_minimize, which fills its stats and keeps the
 *    last state on OFDFT_ENOCONV) and ofdft_last_error() describes it.
 *  - Environment, read by ofdft_setup (diagnostics): OFDFT_DEBUG_SYNC=1
 *    checks every launch and runs loops from the host; OFDFT_NO_GRAPHS=1
 *    runs loops from the host; OFDFT_DLINE_WS="dk,threads" (dk 8 or 16,
 *    threads <= 256, a multiple of 32 dividing 32 dk) starts the context
 *    with the warp-synchronous derivative passes.
 */
#ifndef OFDFT_H
#define OFDFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ofdft_ctx ofdft_ctx;

typedef enum {
    OFDFT_OK = 0,
    OFDFT_EINVAL = -1,    /* bad argument (sizes, cell, temperature, pointer) */
    OFDFT_ENOMEM = -2,    /* device or host allocation failed */
    OFDFT_ENOCONV = -3,   /* minimisation did not reach the tolerance */
    OFDFT_ENUMERIC = -4,  /* NaN/Inf or non-positive density met */
    OFDFT_ETIMEOUT = -5,  /* reserved: a bounded device wait ran out */
    OFDFT_EDEVICE = -6,   /* CUDA error (message in ofdft_last_error) */
    OFDFT_EBUSY = -7,     /* work still in flight (ofdft_minimize_query, ofdft_serve_poll) */
    OFDFT_ECANCELED = -8  /* a served request cancelled by ofdft_serve_cancel */
} ofdft_status;

/* Non-interacting free-energy functional (Table I keywords, Sec. III). */
typedef enum {
    OFDFT_FTTF = 0,   /* KINE TTF: finite-T Thomas-Fermi, Eqs. (TF), (fTF) */
    OFDFT_SGA = 1,    /* KINE HVWTF, PARA MU 5/27: Eq. (SGA-F) */
    OFDFT_VT84F = 2,  /* KINE VT84F: Eq. (VT84F), the "ftGGA" of this library */
    OFDFT_KST2 = 3,   /* KINE KST2: Eq. (KST2F) */
    OFDFT_VWTF = 4,   /* KINE HVWTF, PARA MU 5/3: Sec. III B item (vi) */
    OFDFT_TW = 5,     /* KINE PBETWF: Sec. III B item (iv) */
    OFDFT_APBEF = 6   /* KINE APBEF: Sec. III B item (iii) */
} ofdft_functional;

typedef enum {
    OFDFT_FP64 = 0,   /* every field and reduction in FP64 */
    OFDFT_MIXED = 1   /* FP32 FFTs and pointwise terms, FP64 reductions, line
                         search, Ewald and forces; final energies in FP64 */
} ofdft_precision;

/* Arithmetic of the FP64 field sets' evaluation kernels: the FFTs, the
 * G-space terms and the pointwise functional (f_s, its derivatives and PZ81,
 * Eqs. (FGGA), (vftGGA), (vxc1)), and of the structure factor and local
 * forces (sums over ions, Eq. (M12)).  Fields and spectra stay binary64 in
 * memory, and the reduction totals, CG scalars, Ewald terms and MD stay
 * binary64 either way (the evaluation's block partials add in double-float
 * within a block with F32X2; the CG vector kernels' partials always do,
 * from binary64 per-thread sums; blocks are added in binary64). */
typedef enum {
    OFDFT_PW_F32X2 = 0,  /* double-float pairs on the FP32 units (about 48
                            significant bits): the energy agrees with the
                            binary64 kernels to about 1e-13 relative, the
                            pointwise terms to about 1e-13 of their size;
                            points outside the pointwise routine's range
                            (n outside [1e-18, 1e18], s^2 > 1e10, t outside
                            the tabulated [2^-20, 2^34)) use binary64.
                            Intermediate values keep the binary32 exponent
                            range: a density whose potential passes 3e38
                            (GGA functionals next to n ~ 1e-20) gives
                            OFDFT_ENUMERIC here and needs OFDFT_PW_F64 */
    OFDFT_PW_F64 = 1     /* binary64 throughout the evaluation */
} ofdft_pointwise;

/* Local pseudopotential of the ions (Sec. V A).  Either form drops G = 0;
 * the dropped non-Coulomb constant is reported as ofdft_energy.E_alphaZ. */
typedef enum {
    OFDFT_LPP_GAUSS = 0,  /* Gaussian ion: v(G) = -4 pi Z exp(-G^2 rc^2/4)/(Omega G^2) */
    OFDFT_LPP_HA = 1      /* Heine-Abarenkov, Eq. (E4A): v(q) = -4 pi/(Omega q^2)
                             [(Z - A rc) cos(q rc) + (A/q) sin(q rc)] exp(-(q/qc)^6);
                             one parameter set, so every ion must have the same Z
                             (else OFDFT_EINVAL).  H: rc = 0.25, A = 6.18, qc = 29.97 */
} ofdft_lpp;

typedef struct {
    int xc;           /* 1: Perdew-Zunger LDA XC (Sec. IV, used in Sec. VI); 0: none */
    double rc;        /* local pseudopotential core radius in bohr (both forms; > 0) */
    int precision;    /* ofdft_precision */
    int device;       /* CUDA device ordinal */
    void *stream;     /* cudaStream_t to run on, or NULL for a library stream */
    int pointwise;    /* ofdft_pointwise: arithmetic of the FP64 field sets */
    int lpp;          /* ofdft_lpp */
    double lpp_A;     /* OFDFT_LPP_HA: core depth A in hartree (finite) */
    double lpp_qc;    /* OFDFT_LPP_HA: cutoff wave number qc in 1/bohr (> 0) */
} ofdft_params;

/* Energy partition (Sec. V C sample output) and pressure terms; hartree,
 * hartree/bohr^3.  F_tot = F_s + E_H + E_loc + F_xc + E_ion. */
typedef struct {
    double F_tot;     /* total free energy (QE "free energy Etot") */
    double F_s;       /* non-interacting free energy, Eq. (E4) */
    double minus_TS;  /* non-interacting entropic part -T S_s */
    double E_H;       /* Hartree, Eq. (E2) */
    double E_loc;     /* int n v_ext */
    double F_xc;      /* XC free energy */
    double E_ion;     /* ion-ion (Ewald) energy of Eq. (E1) */
    double E_int;     /* internal energy F_tot + T S_s */
    double mu;        /* chemical potential (Euler equation, Eq. (E10)) */
    double E_alphaZ;  /* dropped G=0 non-Coulomb LPP term, reported only */
    double P;         /* pressure -Tr(Sigma)/3, Eq. (pressure); no ion kinetic part */
    double P_s, P_xc, P_H, P_loc, P_ion;
} ofdft_energy;

typedef struct {
    int iterations;      /* CG iterations (all precisions) */
    int evaluations;     /* energy+potential evaluations (all precisions) */
    double gnorm;        /* final ||dF/dphi|| = (dV sum g^2)^{1/2}, g = 2 phi (v - mu) */
    int status;          /* ofdft_status of the minimisation */
    int evaluations_lo;  /* of which in FP32 (OFDFT_MIXED contexts) */
} ofdft_stats;

typedef struct {
    double dt_fs;       /* time step in femtoseconds */
    double T_kelvin;    /* thermostat temperature; <= 0 switches it off (NVE) */
    double tau_steps;   /* Nose-Hoover period in time steps (Q = g kT tau^2 / 4 pi^2) */
    double gtol;        /* electronic tolerance on ||dF/dphi|| per MD step */
    int maxit;          /* CG iteration cap per MD step */
} ofdft_md_params;

/* Fill *p with defaults: xc = 1, rc = 0.25, FP64, device 0, library stream,
 * double-float pointwise functional, Gaussian LPP (lpp_A = 6.18 and
 * lpp_qc = 29.97, the Eq. (E4A) values for H, for when lpp is switched). */
void ofdft_default_params(ofdft_params *p);

/*
 * Create a context: cell, ions, grid, temperature and functional
 * (Sec. V C, create_ofdftgeom + the PROFESS input of Sec. V B).
 *  cell[9]     rows a, b, c: the lattice vectors in bohr (Cartesian
 *              components).  Orthorhombic (off-diagonals 0, positive
 *              diagonal) or general (triclinic, right-handed: det > 0);
 *              grid point (i, j, k) sits at (i/nx) a + (j/ny) b + (k/nz) c
 *              and G = kx a* + ky b* + kz c* with the reciprocal vectors.
 *              Otherwise OFDFT_EINVAL.  (ofdft_energy_potential_static
 *              takes orthorhombic cells only.)
 *  grid[3]     nx, ny, nz: even, factors in {2,3,5} only, 8 <= n <= 512.
 *  nat, ions   ions[nat][3] Cartesian bohr; Z[nat] valence charges (> 0).
 *  T_kelvin    electron temperature (> 0).
 *  functional  ofdft_functional.
 *  params      NULL for defaults.
 * The density starts uniform, phi = (N_e/Omega)^{1/2}, N_e = sum Z.
 */
ofdft_status ofdft_setup(const double cell[9], const int grid[3], int nat,
                         const double *ions, const double *Z, double T_kelvin,
                         int functional, const ofdft_params *params, ofdft_ctx **out);

/* New ion positions ions[nat][3] (bohr); recomputes v_ext(G) and Ewald terms. */
ofdft_status ofdft_set_positions(ofdft_ctx *ctx, const double *ions);

/* Replace phi by host phi[N] (renormalised to N_e), or by the uniform
 * density if phi is NULL. */
ofdft_status ofdft_set_phi(ofdft_ctx *ctx, const double *phi);

/*
 * One evaluation of F_tot[n] and v = dF/dn at n = phi^2 (Eqs. (E1)-(E4),
 * (vTF) or (vftGGA), (vxc1), (E2)), where phi is host phi[N] or, if NULL,
 * the context's current phi.  Fills *E (may be NULL) and, if v is not NULL,
 * the host array v[N] (hartree).
 */
ofdft_status ofdft_energy_potential(ofdft_ctx *ctx, const double *phi,
                                    ofdft_energy *E, double *v);

/*
 * Minimise F_tot over phi with dV sum phi^2 = N_e by nonlinear CG
 * (Sec. II; the CG details are this library's reading, identical to the
 * oracle's): Polak-Ribiere+ directions projected orthogonal to phi,
 * norm-preserving rotations, derivative line search; stops when
 * ||dF/dphi|| < gtol or after maxit iterations (OFDFT_ENOCONV).
 * Starts from the context's current phi and leaves the minimiser there.
 * The whole minimisation runs on the device (one CUDA graph launch; the host
 * reads the result once).  OFDFT_MIXED contexts first iterate in FP32 until
 * the single-precision floor stalls ||g||, then continue in FP64 to gtol, so
 * the result meets the same tolerance as an FP64 context.
 */
ofdft_status ofdft_minimize(ofdft_ctx *ctx, double gtol, int maxit,
                            ofdft_energy *E, ofdft_stats *stats);

/*
 * The same minimisation by truncated Newton, the alternative to CG that
 * Sec. II names (details are this library's reading, identical to the
 * oracle's minimize_tn): each outer step solves H d = -g on the tangent
 * space of the constraint by an inner CG of at most inner_max steps,
 * truncated when ||r|| <= eta ||g|| or at non-positive curvature; H p is
 * the central difference of the gradient map along p (two evaluations);
 * the step takes the CG's norm-preserving rotation and line search from the
 * Newton angle.  Runs host-driven on the FP64 field set (also for
 * OFDFT_MIXED contexts).  stats->evaluations counts every energy +
 * potential evaluation, *hessian_products (may be NULL) the Hessian
 * products.  gtol > 0, maxit > 0, inner_max > 0 and 0 < eta < 1, else
 * OFDFT_EINVAL; OFDFT_ENOCONV (stats filled, last state kept) when maxit
 * is reached or the line search fails; device scratch: nine fields of N
 * doubles for the duration of the call.
 */
ofdft_status ofdft_minimize_tn(ofdft_ctx *ctx, double gtol, int maxit, int inner_max, double eta,
                               ofdft_energy *E, ofdft_stats *stats, int *hessian_products);

/*
 * ofdft_minimize in two halves, so that many contexts (each on its own
 * stream) minimise concurrently: _start enqueues the whole minimisation on
 * the context's stream and returns at once; _query returns OFDFT_OK once it
 * has finished and OFDFT_EBUSY before; _wait blocks until it has finished and
 * reports as ofdft_minimize does.  Every other call on the context returns
 * OFDFT_EBUSY between _start and _wait.  With OFDFT_DEBUG_SYNC=1 or an active
 * kernel timer _start runs the minimisation to completion itself.
 */
ofdft_status ofdft_minimize_start(ofdft_ctx *ctx, double gtol, int maxit);
ofdft_status ofdft_minimize_query(ofdft_ctx *ctx);
ofdft_status ofdft_minimize_wait(ofdft_ctx *ctx, ofdft_energy *E, ofdft_stats *stats);

/*
 * Batched single-point solves: minimise n independent contexts at once (the
 * uneven-size batch of the library's batched form).  All minimisations are
 * the independent branches of one CUDA graph, launched once on the first
 * context's stream after the work already queued on every context's stream
 * (the executable graph is kept by the first context and reused while the
 * same contexts come in the same order); the solves overlap on the device
 * and each takes exactly the steps it takes alone.  Contexts on different
 * devices, or with host-driven loops (OFDFT_DEBUG_SYNC, kernel timer), run
 * as one graph launch each on their own streams.  E[n] and stats[n]
 * (either may be NULL) receive the results.
 * Returns OFDFT_OK when every solve converged, else the first failing
 * status (all results are still filled).
 */
ofdft_status ofdft_batch_minimize(int n, ofdft_ctx *const *ctxs, double gtol, int maxit,
                                  ofdft_energy *E, ofdft_stats *stats);

/*
 * Device memory a context with this grid, ion count and precision holds
 * (bytes, an upper estimate), for admission control before ofdft_setup.
 */
ofdft_status ofdft_footprint(const int grid[3], int nat, int precision, double *bytes);

/*
 * Autotune the launch shapes of this context's field kernels (pairs of z
 * lines per block of the z passes, column-tile width of the y and x passes):
 * every candidate is timed on this context's grid and the fastest kept.
 * Results are cached per (grid, precision) for the process, so contexts of
 * the same shape reuse them.  reps >= 1 timed evaluations per candidate.
 */
ofdft_status ofdft_autotune(ofdft_ctx *ctx, int reps);

/*
 * Hellmann-Feynman plus Ewald forces at the current density, Eq. (M12):
 * F[nat][3] in hartree/bohr (may be NULL), and the pressure P
 * (hartree/bohr^3, may be NULL).
 */
ofdft_status ofdft_forces(ofdft_ctx *ctx, double *F, double *pressure);

/*
 * Stress tensor at the current density, Eq. (StressTensor):
 * Sigma_ab = (1/V) sum_nu (dF/dh_a,nu) h_b,nu (hartree/bohr^3, row-major
 * sigma[9], symmetric), so that P = -Tr Sigma / 3 (Eq. (pressure)); call it
 * after ofdft_minimize for the equilibrium value.  Terms, for a homogeneous
 * strain at fixed fractional coordinates and V n(G):
 *   non-interacting  delta_ab/V int (f_s - n v_s) - (1/V) int W_a d_b n,
 *                    W = d f_s/d grad n (Eqs. (stressTF_a), (stressTF_b))
 *   XC               delta_ab/V int n (eps_xc - v_xc)   (Eq. (stressLSDAxc))
 *   Hartree          -delta_ab E_H/V + sum_G 4 pi |n(G)|^2 G_a G_b/G^4
 *   local pseudo.    -delta_ab E_loc/V - 2 sum_G Re[n*(G) dv/dG^2] G_a G_b
 *   ions             Ewald stress (real-space pairs, reciprocal sum, background)
 * terms (may be NULL) receives the five tensors in that order ([5][9]).
 * One evaluation plus the stress sums; the density is not changed.
 */
ofdft_status ofdft_stress(ofdft_ctx *ctx, double *sigma, double *terms);

/* Copy the current density n = phi^2 to host n[N]. */
ofdft_status ofdft_get_density(ofdft_ctx *ctx, double *n);

/* Ion masses m[nat] in electron masses (default: hydrogen, 1.00794 u). */
ofdft_status ofdft_set_masses(ofdft_ctx *ctx, const double *m);

/*
 * Advance the MD state by nsteps velocity-Verlet steps with a Nose-Hoover
 * thermostat (the QE integrator of Fig. (P-QE); the paper's runs used an
 * Andersen thermostat).  Each step: thermostat half step, half kick, drift,
 * new v_ext and Ewald terms, density extrapolated as 2 phi_n - phi_{n-1},
 * CG minimisation, forces (Eq. (M12)), half kick, thermostat half step.
 *  pos, vel   [nat][3] in/out on the host (bohr, bohr per atomic time unit),
 *             or NULL to use and keep the device-resident state.  On entry a
 *             pos that differs from the current positions starts a new
 *             trajectory there (thermostat reset, density re-minimised); a
 *             pos equal to them (e.g. what the previous call returned) only
 *             costs the copies.  vel on entry replaces the velocities.  On
 *             return both hold the state after the last step.
 *  F          [nat][3] out (may be NULL); E, stats out (may be NULL).
 * The first call at a new geometry minimises and computes forces first;
 * nsteps = 0 does only that.
 */
ofdft_status ofdft_md_step(ofdft_ctx *ctx, const ofdft_md_params *mp, int nsteps,
                           double *pos, double *vel, double *F,
                           ofdft_energy *E, ofdft_stats *stats);

/*
 * Andersen thermostat (the NVT ensemble of the paper's MD runs, Sec. VI):
 * ion I collides when u[I] < prob and then takes the velocity
 * sqrt(kT/m_I) xi[I], a Maxwell-Boltzmann draw at T_kelvin.  u[nat]
 * (uniform in [0, 1)) and xi[nat][3] (standard normal) are the caller's
 * random numbers, host arrays copied by the call.  Acts on the
 * device-resident MD velocities: run ofdft_md_step with T_kelvin <= 0 (no
 * Nose-Hoover) and pos = vel = NULL between calls, e.g. one call per step
 * with prob = dt / (collision time).  ncoll (may be NULL) receives the
 * number of collisions.  Velocities redrawn this way leave
 * ofdft_md_conserved without meaning.  OFDFT_EINVAL for NULL arrays,
 * T_kelvin <= 0, prob outside [0, 1] or a non-finite xi.
 */
ofdft_status ofdft_md_andersen(ofdft_ctx *ctx, double T_kelvin, double prob, const double *u,
                               const double *xi, int *ncoll);

/* Copy the MD state out: pos, vel [nat][3] (either may be NULL). */
ofdft_status ofdft_md_state(ofdft_ctx *ctx, double *pos, double *vel);

/* Nose-Hoover extended energy K + F_tot + Q xi^2/2 + g kT eta of the last step. */
ofdft_status ofdft_md_conserved(ofdft_ctx *ctx, double *H);

/* Grid size N and the number of ions of a context. */
ofdft_status ofdft_sizes(ofdft_ctx *ctx, long long *N, int *nat);

/*
 * Diagnostics: record CUDA events around every launch of one kernel class on
 * the context's stream (no extra synchronisation).  id: 0 off,
 * 1 pointwise GGA functional, 2 derivative passes along x and y (gradient of
 * n, divergence of W), 4 y pass, 5 z forward pass, 6 z final pass, 7 x pass
 * of the Hartree and local-pseudopotential potential; id + 8 times only the
 * class's FP32 launches, id + 16 only its FP64 ones.  ofdft_timer_read
 * synchronises the stream,
 * returns the summed event time (ms) and the launch count, and optionally
 * clears them.
 */
ofdft_status ofdft_timer_select(ofdft_ctx *ctx, int id);
ofdft_status ofdft_timer_read(ofdft_ctx *ctx, double *total_ms, long long *launches, int reset);

/* Number of CUDA kernels this context has launched since setup. */
long long ofdft_kernel_launches(ofdft_ctx *ctx);

/* Message for the last error on ctx (or of the last failed setup if ctx is
 * NULL).  Valid until the next call on ctx. */
const char *ofdft_last_error(ofdft_ctx *ctx);

/*
 * Host-side evaluation of the tabulated temperature functions used by the
 * kernels (no GPU needed): for each t[i], out[i*8 + k] = xi, zeta, A, B and
 * their t-derivatives, with xi = kappa - t kappa', zeta = -t kappa'
 * (Eq. (xizeta)), A = (h~ - t h~')/xi, B = t h~'/zeta (Eq. (s_s)).
 */
ofdft_status ofdft_tfunc_eval(long long n, const double *t, double *out);

/*
 * Host-side evaluation of the double-float primitives the FP64 field
 * kernels compute with (no GPU needed), for checks against their error
 * bounds.  Each input is first rounded to the nearest double-float (hi =
 * (float)x, lo = (float)(x - hi)); out[i] is the result as a binary64.
 *   op 0  x + y         (Joldes-Muller-Popescu accurate sum)
 *   op 1  x * y         (FMA-based product)
 *   op 2  x / y         (binary32 quotient plus one correction)
 *   op 3  sqrt(x)       x > 0
 *   op 4  exp(x)        x > -87 (0 below)
 *   op 5  e^x - 1       x <= 0
 *   op 6  ln(x)         x > 0, normal binary32 range
 *   op 7  x^(-1/3)      x > 0, normal binary32 range
 * y is read for ops 0-2 only.  OFDFT_EINVAL for a bad op, count or pointer.
 */
ofdft_status ofdft_ffmath_eval(int op, long long count, const double *x, const double *y, double *out);

/*
 * Host-side evaluation of the pointwise functional the field kernels apply
 * (no GPU needed), for checks of its arithmetic.  For each of count points
 * with density n[i] > 0 (bohr^-3) and g2[i] = |grad n|^2, at T_kelvin:
 *   out[6 i + 0] = f_s            free-energy density, Eq. (FGGA) (ftTF: Eq. (fTF))
 *   out[6 i + 1] = T s_s          entropic part tau0 zeta F_sigma
 *   out[6 i + 2] = d f_s / d n    without the divergence term, Eq. (vftGGA)
 *   out[6 i + 3] = W              d f_s / d(grad n) = W grad n
 *   out[6 i + 4] = eps_xc         PZ81 energy per electron (0 when xc = 0)
 *   out[6 i + 5] = v_xc           PZ81 potential (0 when xc = 0)
 * arith: ofdft_pointwise; with OFDFT_PW_F32X2 the double-float routine runs
 * as compiled for the host (same source as the kernels'), falling back to
 * binary64 outside its domain; *n_f2 (optional) receives how many points it
 * handled.  OFDFT_EINVAL for a bad functional, arith, count or pointer.
 */
ofdft_status ofdft_pointwise_eval(int functional, int xc, double T_kelvin, long long count, const double *n,
                                  const double *g2, int arith, double *out, long long *n_f2);

void ofdft_destroy(ofdft_ctx *ctx);

/*
 * Allocation-free energy and potential (the paper has no counterpart; this
 * exists for callers that must not allocate device memory: latency-critical
 * loops, where cudaMalloc may synchronise the whole GPU, and programs whose
 * device memory is owned by another allocator).  It computes what
 * ofdft_setup + ofdft_energy_potential compute (F_tot and its terms, the
 * pressure terms, v = dF/dn at n = phi^2), in FP64, with the same kernels,
 * but every device scratch buffer is carved from one fixed array compiled
 * into the library: about 2.4 MB that each GPU loading the library holds
 * until the process exits.  The call allocates no memory, on the device or
 * the host.
 *  cell[9], grid[3], nat, ions, Z, T_kelvin, functional: as ofdft_setup,
 *              but orthorhombic cells only (else OFDFT_EINVAL).
 *  xc, rc: as ofdft_params (Gaussian ion only).
 *  phi_dev  device pointer, N doubles (input; not modified), 16-byte aligned.
 *  v_dev    device pointer, N doubles (output potential), 16-byte aligned;
 *           also the call's scratch for one field before v is written.
 *  E        host output (may be NULL).
 *  stream   cudaStream_t to run on, or NULL for the default stream; the call
 *           returns after the stream has finished its work.
 * Limits: each grid edge even, {2,3,5}-smooth and at most 64;
 * nx*ny*nz <= 32768; 1 <= nat <= 64.  Anything larger returns OFDFT_EINVAL,
 * as do Z <= 0, non-finite positions, T or rc.
 * No call may be made on a stream that is being captured (the call copies
 * from pageable host memory and synchronises): OFDFT_EINVAL.  The first
 * call on a device does a one-time set-up on the current device (looks up
 * the array's device address, uploads the temperature table).  The set-up
 * runs under a mutex, so
 * first calls from several host threads are safe on the host.  It is cached
 * for the life of the device's context: after cudaDeviceReset (or a release
 * of the primary context) the cached address and table are stale and the
 * path must not be called again in that process.  All calls share the array
 * and it keeps the last call's contents: calls that overlap on the GPU (from
 * other threads or streams) race, so serialise them.
 */
ofdft_status ofdft_energy_potential_static(const double cell[9], const int grid[3], int nat,
                                           const double *ions, const double *Z, double T_kelvin,
                                           int functional, int xc, double rc,
                                           const double *phi_dev, double *v_dev,
                                           ofdft_energy *E, void *stream);

/*
 * Serving: a request loop for equation-of-state points.  Each request is
 * one system (cell, ions, grid, temperature, functional, precision) and a
 * number of MD steps; requests queue in arrival order and are admitted while
 * a slot is free and the request's device footprint (ofdft_footprint) fits
 * in the memory budget.  A queued request that does not fit yet may be
 * passed by up to max_bypass later requests that do; after that nothing is
 * admitted ahead of it until it fits.  An admitted request gets its own context and
 * stream, so requests arriving while others run overlap with them on the
 * device (continuous batching), and each keeps its density, CG state and FFT
 * tables resident until it finishes.  Contexts are independent, so a
 * request's results do not depend on what else runs.
 */
typedef struct ofdft_server ofdft_server;

typedef struct {
    int device;               /* CUDA device ordinal */
    int max_slots;            /* requests running at once (worker threads), >= 1 */
    double hbm_budget_bytes;  /* admission budget; <= 0: 90% of the device memory free at start */
    int dry_run;              /* 1: no device work, each request sleeps dry_run_ms in md_steps + 1
                                 equal parts (host tests) */
    double dry_run_ms;
    int max_bypass;           /* >= 0: how many later requests may be admitted ahead of a queued
                                 request that does not fit yet (0: strict arrival order) */
} ofdft_serve_params;

typedef struct {
    double cell[9];           /* as ofdft_setup */
    int grid[3];
    int nat;
    const double *ions;       /* [nat][3], copied at submit */
    const double *Z;          /* [nat], copied at submit */
    const double *vel;        /* [nat][3] initial velocities or NULL (zero), copied */
    double T_kelvin;          /* electron temperature and thermostat temperature */
    int functional;           /* ofdft_functional */
    int precision;            /* ofdft_precision */
    int xc;
    double rc;
    int md_steps;             /* MD steps after the initial minimisation (>= 0) */
    double dt_fs;
    double gtol;
    int maxit;
} ofdft_request;

typedef struct {
    long long id;
    int status;               /* ofdft_status of the request */
    ofdft_energy E;           /* after the last step */
    double P_mean;            /* mean pressure over the MD steps (or the single point) */
    int steps_done;           /* MD steps completed (0 if the initial minimisation failed) */
    long long evaluations;    /* energy+potential evaluations, all steps */
    double t_submit, t_admit, t_done;   /* seconds on the server clock (t_admit -1 for a
                                           request cancelled while queued) */
    double footprint_bytes;
} ofdft_result;

ofdft_status ofdft_serve_start(const ofdft_serve_params *p, ofdft_server **out);
/* Queue a request; *id receives its id.  OFDFT_ENOMEM if its footprint
 * exceeds the whole budget, OFDFT_EINVAL for bad sizes. */
ofdft_status ofdft_serve_submit(ofdft_server *s, const ofdft_request *r, long long *id);
/* OFDFT_OK and *res filled once request id has finished, OFDFT_EBUSY while
 * it is queued or running, OFDFT_EINVAL for an unknown id. */
ofdft_status ofdft_serve_poll(ofdft_server *s, long long id, ofdft_result *res);
/* Cancel request id.  A queued request is removed at once and finishes with
 * status OFDFT_ECANCELED and no steps; a running one stops before its next
 * MD step (the initial minimisation or a step already started runs to its
 * end) and finishes with OFDFT_ECANCELED, the steps it completed, and the
 * energy and mean pressure of those.  OFDFT_OK also for a request that has
 * already finished (its result is unchanged); OFDFT_EINVAL for an unknown
 * id. */
ofdft_status ofdft_serve_cancel(ofdft_server *s, long long id);
/* Block until every submitted request has finished (timeout_s <= 0: no limit;
 * OFDFT_ETIMEOUT when it runs out). */
ofdft_status ofdft_serve_drain(ofdft_server *s, double timeout_s);
/* Seconds since ofdft_serve_start on the server clock (steady). */
double ofdft_serve_clock(ofdft_server *s);
/* Peak bytes of admitted footprints and peak concurrent requests so far. */
ofdft_status ofdft_serve_peaks(ofdft_server *s, double *bytes, int *running);
/* Finish queued and running requests, join the workers, free the server. */
ofdft_status ofdft_serve_stop(ofdft_server *s);

#ifdef __cplusplus
}
#endif
#endif /* OFDFT_H */
