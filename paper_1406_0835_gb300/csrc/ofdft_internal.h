// Internal declarations shared by the CUDA translation units of libofdft.
// Not part of the public C ABI (see include/ofdft.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ofdft.h"

namespace ofdft {

// ----------------------------------------------------------------- complex
template <typename T> struct CT;
template <> struct CT<double> { typedef double2 type; };
template <> struct CT<float> { typedef float2 type; };
template <typename T> using cplx = typename CT<T>::type;

template <typename C> __host__ __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b)
{
    C r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b)
{
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmk<C>(a.x * s, a.y * s); }
// multiply by -i (forward sign) or +i (inverse sign)
template <typename C, bool INV> __host__ __device__ __forceinline__ C cmuli(C a)
{
    return INV ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

// ------------------------------------------------------------ FFT plans
constexpr int kMaxStages = 16;

// One axis of a 3D transform: a mixed-radix Stockham schedule and a
// twiddle table w[m] = exp(-2 pi i m / n), m = 0..n-1, in device memory.
struct FftAxis {
    int n;
    int nst;
    int rad[kMaxStages];
    int ns[kMaxStages];      // product of the radices before each stage
    const void *tw;          // cplx<T>[n]
};

// Geometry of the periodic orthorhombic grid, C order [ix][iy][iz], and of
// the half spectrum [ix][iy][kz], kz = 0..nz/2.
struct GridInfo {
    int nx, ny, nz, K;
    long long N, NH;
    double Lx, Ly, Lz, omega, dV;
    double rc;               // Gaussian local pseudopotential radius
    double bx, by, bz;       // reciprocal spacing 2 pi / L per axis
    int zP;                  // z passes: line pairs per block (0: default rule)
    int tk;                  // y/x passes: half-spectrum columns per tile (4, 8 or 16)
};

inline void grid_reciprocal(GridInfo &g)
{
    if (g.tk <= 0) g.tk = 8;
    const double tp = 6.283185307179586477;
    g.bx = tp / g.Lx;
    g.by = tp / g.Ly;
    g.bz = tp / g.Lz;
}

// Tabulated temperature functions xi, zeta, A, B of t (see tfunc_table.cpp).
constexpr int kTfDeg = 10;                 // polynomial degree per panel
constexpr int kTfNc = kTfDeg + 1;
constexpr int kTfSub = 4;                  // panels per octave of t
constexpr int kTfEmin = -20;               // t range [2^kTfEmin, 2^kTfEmax)
constexpr int kTfEmax = 34;
constexpr int kTfPanels = (kTfEmax - kTfEmin) * kTfSub;
constexpr int kTfFuncs = 4;                // xi, zeta, A, B
constexpr int kTfSize = kTfPanels * kTfFuncs * kTfNc;

// Build the table on the host (FP64 monomial coefficients per panel).
const std::vector<double> &tfunc_table_host();
// The same table written into caller storage of kTfSize doubles.
void tfunc_table_fill(double *tab);

// Functional selector and constants for the enhancement factors.
struct FuncParams {
    int kind;       // 0 ftTF, 1 SGA-form (mu), 2 VT84F, 3 KST2-form (C1, a1)
    double p0, p1;  // mu | C1, a1
};
FuncParams functional_params(int functional);

// Device-resident state of one CG minimisation (reading R9 of the paper's
// unstated CG details).  Reductions write the sums; single-thread controller
// kernels turn them into the scalars the vector kernels read, and drive the
// graph's conditional loops.
struct CgState {
    // configuration (written by the host before a minimisation)
    double gtol, dV, ls_tol, theta0, Ne;
    double switch_g;   // stagnate mode: also stop once ||g|| < switch_g (0: off)
    int maxit, max_ls, stagnate;
    int pad0;
    // reduction outputs
    double ev[18];     // evaluation: E_H, E_loc, P_loc, GGA sums [3..8], final sums [9..17]
    double rg[2];      // sum g^2, sum g.g_prev
    double rd[5];      // sum phi.d, d.d, d.g, phi.phi, phi.g
    double rh[1];      // sum 2 phi v dhat
    double rn[1];      // sum phi^2
    // iteration state
    double mu, gg, ggprev, gnorm, beta, c1, c2, D0, theta_prev, scale;
    double cs[2];      // cos, sin of the trial angle (read by the evaluation kernels)
    double th, lo, Dlo, hi, Dhi, pa, Da;
    double best_g;
    double c12r[3];    // c1, c2, restart (read by the direction kernel)
    int best_it, restart, have_prev, it, nevals, nls, ls_active, accepted, status, done, fallback;
    int nouter;        // executions of the iteration body (directions built)
    double ev_acc[18]; // evaluation sums at the last accepted point
};

// Status codes of CgState::status (besides ofdft_status values).
constexpr int kCgStagnated = 1;   // stopped at the precision floor (stagnate mode)

// Reduction quantities (indices into the scalar block).
enum Quantity {
    Q_FS = 0,      // sum f_s
    Q_TS,          // sum tau0 zeta F_sigma (T S density)
    Q_FXC,         // sum n eps_xc
    Q_PS,          // sum (n df/dn - f)
    Q_WG,          // sum W . grad n
    Q_PXC,         // sum n (v_xc - eps_xc)
    Q_PHI2V,       // sum phi^2 v
    Q_PHI2,        // sum phi^2
    Q_DTH,         // sum 2 phi v dphi/dtheta
    Q_EH,          // Hartree energy (already scaled)
    Q_ELOC,        // local pseudopotential energy (scaled)
    Q_PLOC,        // LPP pressure (scaled)
    Q_COUNT_EVAL,
};

}  // namespace ofdft
