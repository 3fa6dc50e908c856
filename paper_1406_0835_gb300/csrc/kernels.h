// Host-side launchers of the libofdft kernels (templated on the field type).
#pragma once

#include "ofdft_internal.h"

namespace ofdft {

// ---- grid fields (kernels_fields.cu)
// z pass, forward: n = phi^2 (mode 1), the trial rotation phi cos + dhat sin
// written to phit (mode 2) or a plain field (mode 0), R2C along z into the
// half spectrum out; with dz also d_z n into the real field dz.
template <typename T>
void launch_zfwd(const GridInfo &g, const FftAxis &az, int mode, const T *in, const T *phi,
                 const T *dhat, T c, T s, const void *cs, T *phit, cplx<T> *out, cudaStream_t st,
                 T *dz = nullptr);
// Derivative of a real field along grid axis 0 (x) or 1 (y) by 1-D
// transforms along that axis: out (= or, acc != 0, +=) d f, f = phi^2 for
// mode 0 and f = in for mode 1 (scale GridInfo::ds).
template <typename T>
void launch_dline(const GridInfo &g, const FftAxis &fa, int axis, int mode, int acc, const T *in, T *out,
                  cudaStream_t st);
// Pointwise functional + XC: reads phi and the derivatives of n in d0..d2,
// writes v_part and, over d0..d2, the fields U_j whose derivatives sum to
// div W.  Partials: 6 rows (12 with stress: sum W_a d_b n in rows 6..11, FP64
// sets only) of the returned number of columns.
template <typename T>
int launch_pw(const GridInfo &g, T *d0, T *d1, T *d2, const T *phit, T temp, const FuncParams &fp, const T *tab,
              int xc, T *vpart, double *part, bool stress, cudaStream_t st);
// z pass, final (ftTF): C2R of v_HL, pointwise functional, potential and sums.
template <typename T>
int launch_zfinal(const GridInfo &g, const FftAxis &az, bool fttf, const cplx<T> *dspec,
                  const T *vpart, const T *phit, const T *phi, const T *dhat, T c, T s,
                  const void *cs, T temp, const FuncParams &fp, const T *tab, int xc, T *vout,
                  double *part, cudaStream_t st);
// z pass, final (GGA): v = v_HL - d_z U_z + v_part - div - div2 (div may
// alias vout; div2 may be null).
template <typename T>
int launch_zfinal_gga(const GridInfo &g, const FftAxis &az, const cplx<T> *dspec, const T *uz, const T *vpart,
                      const T *div, const T *div2, const T *phit, const T *phi, const T *dhat, T c, T s,
                      const void *cs, T *vout, double *part, cudaStream_t st);
template <typename T>
void launch_ypass(const GridInfo &g, const FftAxis &ay, bool inv, cplx<T> *data, int nfields,
                  long long fstride, cudaStream_t st);
template <typename T>
int launch_xhl(const GridInfo &g, const FftAxis &ax, cplx<T> *spec, const cplx<T> *vext,
               cplx<T> *nG_out, int inverse, double *part, cudaStream_t st);
size_t field_smem_max(const GridInfo &g, size_t csize);
// blocks (and partial sums per quantity) of the x passes
int xpass_blocks(const GridInfo &g);
// Largest block the transform kernels were built for.
int fft_max_threads();
template <typename T> cudaError_t set_field_smem_limits(size_t bytes);

// ---- vectors, reductions, ions (kernels_misc.cu)
// Sum part[q * nblk + b] over b for q < nq into out[q] (one block per q, fixed order).
void launch_reduce(const double *part, int nblk, int nq, double *out, cudaStream_t st);
// The three reductions of an evaluation in one launch: rows 0..2 of pA (na
// columns) into out[0..2], rows 0..5 of pB (nb columns, GGA only) into
// out[3..8], rows 0..8 of pC (nc columns) into out[9..17].
void launch_reduce_eval(const double *pA, int na, const double *pB, int nb, const double *pC, int nc, bool gga,
                        double *out, cudaStream_t st);
template <typename T> void launch_fill(long long n, T *x, T val, cudaStream_t st);
template <typename T> void launch_scale(long long n, T *x, double s, const double *sp, cudaStream_t st);
// if *accepted: phi <- phit, v <- vt, gprev <- g; then g = 2 phi (v - *mup);
// part: sum g^2, sum g.gprev (returns blocks)
template <typename T>
int launch_cg_update(long long n, const int *accepted, T *phi, const T *phit, T *v, const T *vt,
                     const double *mup, T *g, T *gprev, double *part, cudaStream_t st);
template <typename T, typename U> void launch_convert(long long n, const T *x, U *y, cudaStream_t st);
// sum x^2 -> part (returns blocks)
template <typename T> int launch_sumsq(long long n, const T *x, double *part, cudaStream_t st);
// y = 2 x - xp; part: sum y^2
template <typename T>
int launch_extrap(long long n, const T *x, const T *xp, T *y, double *part, cudaStream_t st);
// part <- block sums of a.b (returns blocks); out = alpha x + beta y
template <typename T> int launch_dot(long long n, const T *a, const T *b, double *part, cudaStream_t st);
template <typename T>
void launch_axpby(long long n, double alpha, const T *x, double beta, const T *y, T *out, cudaStream_t st);
// g = 2 phi (v - mu); part: sum g^2, sum g.gprev
template <typename T>
int launch_cg_grad(long long n, const T *phi, const T *v, double mu, const double *mup, T *g,
                   const T *gprev, double *part, cudaStream_t st);
// d = -g + beta d; part: sum phi d, sum d^2, sum d g, sum phi^2, sum phi g
template <typename T>
int launch_cg_dir(long long n, const T *g, T *d, double beta, const double *betap, const T *phi,
                  double *part, cudaStream_t st);
// restart: d = -g; else d -= c1 phi; dhat = c2 d; part: sum 2 phi v dhat
template <typename T>
int launch_cg_dhat(long long n, const T *g, T *d, const T *phi, const T *v, double c1, double c2,
                   int restart, const double *c12r, T *dhat, double *part, cudaStream_t st);

// Double-float copies of the phase tables (16 bytes per complex entry, the
// size of a double2): xT[ix][I], yT[iy][I], zT[kz][I] (atoms fastest) and
// zd[I][kz].
struct PhaseTablesDD {
    double2 *xT, *yT, *zT, *zd;
};
// Per-ion axis phase tables exp(-i G_a R_a) for a = x, y, z (complex double,
// [nat][nx], [nat][ny], [nat][K]); with dd also their double-float copies.
void launch_phases(const GridInfo &g, int nat, const double *R, double2 *px, double2 *py,
                   double2 *pz, const PhaseTablesDD *dd, cudaStream_t st);
// v_ext(G) on the half spectrum, Hermitian-symmetrised on Nyquist planes:
// sums over atoms in double-float when dd is given and the grid computes in
// double-float, else binary64.  (A single-precision copy is made with
// launch_convert.)
void launch_vext(const GridInfo &g, int nat, const double *Z, const double2 *px,
                 const double2 *py, const double2 *pz, const PhaseTablesDD *dd, double2 *vext, cudaStream_t st);
// Local-pseudopotential forces from n(G): part[(I * nchunk + c) * 3 + a];
// returns nchunk (= lpp_force_chunks(g, nat, dd != nullptr)).  cn is
// scratch of NH double2.  Double-float sums as launch_vext.
template <typename T>
int launch_lpp_forces(const GridInfo &g, int nat, const double *Z, const double2 *px,
                      const double2 *py, const double2 *pz, const PhaseTablesDD *dd, const cplx<T> *nG,
                      double2 *cn, double *part, cudaStream_t st);
int lpp_force_chunks(const GridInfo &g, int nat, bool dd);
// Chunks of the double-float force kernel for nx * ny = rows (footprints).
int lpp_force_chunks_dd(long long rows, int nat);
// Sum force partials over chunks into F[nat][3] (+= if accumulate).
void launch_force_reduce(int nat, int nchunk, const double *part, double *F, int accumulate,
                         cudaStream_t st);

// The cell of the Ewald real-space sums: rows a_j of a (bohr), ai = a^-1;
// tri = 0 for an orthorhombic cell (a diagonal).
struct EwCell {
    double a[9], ai[9];
    int tri;
};

// Ewald: real-space part per ion -> eparts[nat], F[nat][3];
// reciprocal part over the G list -> S[nG], energy partials, forces added.

void launch_ewald_real(int nat, const double *R, const double *Z, const EwCell &cl, double alpha,
                       double rcut, int3 nimg, double *eion, double *F, cudaStream_t st);
int launch_ewald_recip(int nat, const double *R, const double *Z, int nG, const double *Gv,
                       const double *wG, double2 *S, double *epart, double *F, cudaStream_t st);

// MD: half step A (thermostat half, kick, drift) and B (kick, thermostat half).
void launch_md_a(int nat, const double *m, double *R, double *V, const double *F, double dt,
                 double kT, double Q, int ndof, int thermo, double *nh, cudaStream_t st);
void launch_md_b(int nat, const double *m, double *V, const double *F, double dt, double kT,
                 double Q, int ndof, int thermo, double *nh, cudaStream_t st);
void launch_andersen(int nat, const double *m, double *V, double kT, double prob, const double *u,
                     const double *xi, double *nh, cudaStream_t st);
// Stress tensor parts: Hartree and LPP sums over the half spectrum (12
// partial rows, nx ny columns; returns the column count), and the Ewald
// real-space (6 rows, nat columns) and reciprocal (7 rows; returns the
// column count) sums.
int launch_gstress(const GridInfo &g, int nat, const double *Z, const double2 *px, const double2 *py,
                   const double2 *pz, const PhaseTablesDD *dd, const double2 *nG, double *part, cudaStream_t st);
int launch_ewald_stress(int nat, const double *R, const double *Z, const EwCell &cl, double alpha, double rcut,
                        int3 nimg, int nG, const double *Gv, const double *wG, const double2 *S,
                        double *preal, double *precip, cudaStream_t st);

// ---- device CG controller (cg_control.cu); single-thread kernels.
// use_cond = 0 outside a graph (the handles are then ignored).
void launch_ctl_norm(CgState *s, cudaStream_t st);
void launch_ctl_init(CgState *s, cudaStream_t st);
void launch_ctl_grad(CgState *s, int first, cudaGraphConditionalHandle outer, int use_cond,
                     cudaStream_t st);
void launch_ctl_dir(CgState *s, cudaStream_t st);
void launch_ctl_dhat(CgState *s, cudaGraphConditionalHandle ls, int use_cond, cudaStream_t st);
void launch_ctl_ls(CgState *s, cudaGraphConditionalHandle ls, int use_cond, cudaStream_t st);

}  // namespace ofdft
