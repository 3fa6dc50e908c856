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
    int tws[kMaxStages];     // twiddle stride n / (ns * rad)
    const void *tw;          // cplx<T>[n]
    const void *twf;         // FP64 sets: the same twiddles as double-float pairs (ff::cf2[n])
    int mp;                  // the largest power-of-two radix of the schedule (4 or 8)
};

// Stockham schedule of one axis: radix-8 stages first, then 4, 2, 3, 5;
// max_pow2 (8 or 4) caps the power-of-two radices only (2, 3 and 5 always
// take part, so every {2,3,5}-smooth n factors completely).
inline FftAxis fft_axis(int n, const void *tw, int max_pow2 = 8)
{
    FftAxis a{};
    a.n = n;
    int m = n, ns = 1, k = 0;
    for (int r : {8, 4, 2, 3, 5}) {
        if ((r == 8 || r == 4) && r > max_pow2) continue;
        while (m % r == 0 && k < kMaxStages) {
            a.rad[k] = r;
            a.ns[k] = ns;
            a.tws[k] = n / (ns * r);
            ns *= r;
            m /= r;
            ++k;
        }
    }
    a.nst = k;
    a.tw = tw;
    a.mp = max_pow2;
    return a;
}

// Geometry of the periodic orthorhombic grid, C order [ix][iy][iz], and of
// the half spectrum [ix][iy][kz], kz = 0..nz/2.
struct GridInfo {
    int nx, ny, nz, K;
    long long N, NH;
    double Lx, Ly, Lz, omega, dV;
    double rc;               // local pseudopotential core radius
    int lpp;                 // 0 Gaussian ion, 1 Heine-Abarenkov (Eq. (E4A))
    double ha_A, ha_qc, ha_Z;   // Heine-Abarenkov depth, cutoff and the common ion charge
    double bx, by, bz;       // reciprocal spacing 2 pi / L per axis
    double invN, hr;         // 1 / N, rc^2 / 2
    float bxf, byf, bzf, invNf, hrf;   // the same in FP32 (for the FP32 kernels)
    int zP;                  // z passes: line pairs per block (0: default rule)
    int tk;                  // y/x passes: half-spectrum columns per tile (4, 8 or 16)
    int zth, xth;            // threads per block of the z and of the y/x passes (0: default rule)
    int dk, dth;             // derivative passes: pair columns per tile (4, 8 or 16) and threads (0: default)
    int dws;                 // derivative passes with warp-owned lines (stages synchronised per warp)
    int dd;                  // FP64 fields: FFT and G-space arithmetic in double-float
    float bx2[2], by2[2], bz2[2], invN2[2], hr2[2];   // the same constants as double-float pairs
    // general (triclinic) cell: tri = 1 when the lattice vectors a_j (rows of
    // Am) are not along the axes.  G = kx b_0 + ky b_1 + kz b_2 with
    // a_i . b_j = 2 pi delta_ij; Bm[3 j + c] = component c of b_j; fractional
    // coordinates s = r Ainv.  (Orthorhombic: Bm diagonal = bx, by, bz.)
    int tri;
    double Am[9], Bm[9], Ainv[9];
    float Bmf[9], Bm2[9][2];
    // derivative passes: multiplier scale per grid axis j including the 1/n_j
    // of the 1-D inverse transform: b_j / n_j in an orthorhombic cell (the
    // pass yields the Cartesian derivative), 1 / n_j in a general cell (the
    // lattice-direction derivative, combined with Bm pointwise)
    double ds[3];
    float dsf[3], ds2[3][2];
};

// Derived quantities of a grid (call after setting sizes, cell and rc).
// An orthorhombic grid needs Lx, Ly, Lz; a triclinic one (tri = 1) also Am.
inline void grid_reciprocal(GridInfo &g)
{
    if (g.tk <= 0) g.tk = 8;
    if (g.dk <= 0) g.dk = 4;
    const double tp = 6.283185307179586477;
    if (!g.tri) {
        for (int k = 0; k < 9; ++k) g.Am[k] = 0.0;
        g.Am[0] = g.Lx;
        g.Am[4] = g.Ly;
        g.Am[8] = g.Lz;
    }
    {
        // inverse of Am by cofactors; Bm = 2 pi Ainv^T
        const double *a = g.Am;
        const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                           a[2] * (a[3] * a[7] - a[4] * a[6]);
        double inv[9] = {a[4] * a[8] - a[5] * a[7], a[2] * a[7] - a[1] * a[8], a[1] * a[5] - a[2] * a[4],
                         a[5] * a[6] - a[3] * a[8], a[0] * a[8] - a[2] * a[6], a[2] * a[3] - a[0] * a[5],
                         a[3] * a[7] - a[4] * a[6], a[1] * a[6] - a[0] * a[7], a[0] * a[4] - a[1] * a[3]};
        for (int k = 0; k < 9; ++k) g.Ainv[k] = inv[k] / det;
        for (int j = 0; j < 3; ++j)
            for (int c = 0; c < 3; ++c) g.Bm[3 * j + c] = tp * g.Ainv[3 * c + j];
    }
    g.bx = tp / g.Lx;
    g.by = tp / g.Ly;
    g.bz = tp / g.Lz;
    if (!g.tri) {   // exactly the per-axis spacings
        for (int k = 0; k < 9; ++k) g.Bm[k] = 0.0;
        g.Bm[0] = g.bx;
        g.Bm[4] = g.by;
        g.Bm[8] = g.bz;
    }
    for (int k = 0; k < 9; ++k) {
        g.Bmf[k] = (float)g.Bm[k];
        g.Bm2[k][0] = (float)g.Bm[k];
        g.Bm2[k][1] = (float)(g.Bm[k] - (double)g.Bm2[k][0]);
    }
    g.invN = 1.0 / (double)g.N;
    g.hr = 0.5 * g.rc * g.rc;
    const double dc[5] = {g.bx, g.by, g.bz, g.invN, g.hr};
    float *pc[5] = {g.bx2, g.by2, g.bz2, g.invN2, g.hr2};
    for (int i = 0; i < 5; ++i) {
        pc[i][0] = (float)dc[i];
        pc[i][1] = (float)(dc[i] - (double)pc[i][0]);
    }
    g.bxf = (float)g.bx;
    g.byf = (float)g.by;
    g.bzf = (float)g.bz;
    g.invNf = (float)g.invN;
    g.hrf = (float)g.hr;
    const int na[3] = {g.nx, g.ny, g.nz};
    const double ba[3] = {g.bx, g.by, g.bz};
    for (int j = 0; j < 3; ++j) {
        g.ds[j] = (g.tri ? 1.0 : ba[j]) / (double)na[j];
        g.dsf[j] = (float)g.ds[j];
        g.ds2[j][0] = (float)g.ds[j];
        g.ds2[j][1] = (float)(g.ds[j] - (double)g.ds2[j][0]);
    }
}

// The FP64 or FP32 copy of a grid constant, for kernels templated on A.
template <typename A> __host__ __device__ __forceinline__ A gsel(double d, float f);
template <> __host__ __device__ __forceinline__ double gsel<double>(double d, float) { return d; }
template <> __host__ __device__ __forceinline__ float gsel<float>(double, float f) { return f; }

// Tabulated temperature functions xi, zeta, A, B of t (see tfunc_table.cpp).
constexpr int kTfDeg = 10;                 // polynomial degree per panel
constexpr int kTfNc = kTfDeg + 1;
constexpr int kTfSub = 4;                  // panels per octave of t
constexpr int kTfEmin = -20;               // t range [2^kTfEmin, 2^kTfEmax)
constexpr int kTfEmax = 34;
constexpr int kTfPanels = (kTfEmax - kTfEmin) * kTfSub;
constexpr int kTfFuncs = 4;                // xi, zeta, A, B
constexpr int kTfSize = kTfPanels * kTfFuncs * kTfNc;

// VT84F enhancement factor F(x), x = s^2 (Eq. (VT84F)), as a table of
// G = (F - 1)/x for the double-float kernels: 16 panels per octave of x
// over [2^-20, 2^6), degree 10 in the panel variable u in [-1, 1) (below:
// the quadratic series of F, above: the closed form 5x/3 + 1/x, where
// e^(-alpha x) < 1e-36).
constexpr int kEnDeg = 10;
constexpr int kEnNc = kEnDeg + 1;
constexpr int kEnSub = 16;
constexpr int kEnEmin = -20;
constexpr int kEnEmax = 6;
constexpr int kEnPanels = (kEnEmax - kEnEmin) * kEnSub;
constexpr int kEnSize = kEnPanels * kEnNc;
// Storage of the FP64 field sets' tables, in doubles: the binary64
// temperature table, its double-float split, the enhancement table's split.
constexpr int kDdTabSize = 2 * kTfSize + kEnSize;

// Build the table on the host (FP64 monomial coefficients per panel).
const std::vector<double> &tfunc_table_host();
// The enhancement table (binary64 monomial coefficients, kEnSize doubles).
void enh_table_fill(double *tab);
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
    double e_tol;      // line search: reject trials whose energy rises above
                       // E0 + 1e-4 theta D0 + e_tol |E0| (0: off)
    int maxit, max_ls, stagnate;   // stagnate: window in iterations (0: off)
    int eoff;          // index in ev[] of the F_s sum (F_xc follows two later)
    // reduction outputs
    double ev[18];     // evaluation: E_H, E_loc, P_loc, GGA sums [3..8], final sums [9..17]
    double rg[2];      // sum g^2, sum g.g_prev
    double rd[5];      // sum phi.d, d.d, d.g, phi.phi, phi.g
    double rh[1];      // sum 2 phi v dhat
    double rn[1];      // sum phi^2
    // iteration state
    double mu, gg, ggprev, gnorm, beta, c1, c2, D0, theta_prev, scale;
    double cs[2];      // cos, sin of the trial angle (read by the FP64 evaluation kernels)
    float csf[2];      // the same for the FP32 kernels
    double th, lo, Dlo, hi, Dhi, pa, Da;
    double E0;         // electronic energy at theta = 0 of the current line search
    int hi_nod;        // the upper bracket came from the energy test, not from D > 0
    double best_g;
    double c12r[3];    // c1, c2, restart (read by the direction kernel)
    int best_it, restart, have_prev, it, nevals, nls, ls_active, accepted, status, done, fallback;
    int nouter;        // executions of the iteration body (directions built)
    double ev_acc[18]; // evaluation sums at the last accepted point
};

// Status codes of CgState::status (besides ofdft_status values).
constexpr int kCgStagnated = 1;   // stopped at the precision floor (stagnate mode)
// Stagnate mode: the stage stops when ||g|| has not fallen by 10 % in this
// many iterations.
constexpr int kStagnateIts = 40;

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
