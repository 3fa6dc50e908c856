// Grid-field kernels of one energy + potential evaluation.
//
// A real field is transformed in three passes: z (real-to-complex, two real
// lines packed in one complex line), y and x (complex, on column tiles of
// the half spectrum [ix][iy][kz]).  The G-space work (Hartree, local
// pseudopotential, i G n(G), i G.W(G)) is fused into the x pass and the
// pointwise functional into the z pass, so one GGA evaluation is
//   zfwd(n = phi^2) -> y -> x[grad] -> y^-1 (3) -> z[pointwise, W] -> y (3)
//   -> x[div] -> y^-1 -> z^-1[potential, reductions]
// (ftTF: zfwd -> y -> x[v_HL] -> y^-1 -> z^-1[pointwise, potential]).
//
// Every kernel is written once for a precision tag PR: float and double
// compute in their own type; DD keeps the fields in binary64 in memory and
// computes in double-float (ffmath.cuh) in registers and shared memory, so
// the FP64 path runs on the FP32 units.  KT<PR> names the types.
#include <algorithm>
#include <type_traits>

#include "fft_core.cuh"
#include "kernels.h"
#include "pointwise.cuh"

namespace ofdft {

namespace {

struct DD {};

template <typename PR> struct KT {
    typedef PR T;          // stored real
    typedef cplx<PR> C;    // stored complex
    typedef cplx<PR> CC;   // computed complex (shared memory)
    typedef PR R;          // computed real (and per-thread accumulator)
};
template <> struct KT<DD> {
    typedef double T;
    typedef double2 C;
    typedef ff::cf2 CC;
    typedef ff::f2 R;
};

template <typename PR> constexpr bool is_dd() { return std::is_same<PR, DD>::value; }

// loads and stores between the stored and the computed types; constants
template <typename PR> __device__ __forceinline__ typename KT<PR>::R ldr(typename KT<PR>::T x) { return x; }
template <> __device__ __forceinline__ ff::f2 ldr<DD>(double x) { return ff::split_int(x); }
template <typename PR> __device__ __forceinline__ typename KT<PR>::T str(typename KT<PR>::R x) { return x; }
template <> __device__ __forceinline__ double str<DD>(ff::f2 x) { return ff::to_double(x); }
template <typename PR> __device__ __forceinline__ typename KT<PR>::CC ldc(typename KT<PR>::C v) { return v; }
template <> __device__ __forceinline__ ff::cf2 ldc<DD>(double2 v)
{
    ff::cf2 r;
    r.x = ff::split_int(v.x);
    r.y = ff::split_int(v.y);
    return r;
}
template <typename PR> __device__ __forceinline__ typename KT<PR>::C stc(typename KT<PR>::CC v) { return v; }
template <> __device__ __forceinline__ double2 stc<DD>(ff::cf2 v)
{
    return make_double2(ff::to_double(v.x), ff::to_double(v.y));
}
// grid constant in the computed type (binary64 value d, binary32 copy f,
// double-float pair p)
template <typename PR>
__device__ __forceinline__ typename KT<PR>::R gcst(double d, float f, const float *) { return gsel<PR>(d, f); }
template <> __device__ __forceinline__ ff::f2 gcst<DD>(double, float, const float *p) { return ff::f2(p[0], p[1]); }
constexpr double kFourPi = 12.566370614359172954;
template <typename PR> __device__ __forceinline__ typename KT<PR>::R fourpi() { return (typename KT<PR>::R)kFourPi; }
template <> __device__ __forceinline__ ff::f2 fourpi<DD>()
{
    constexpr ff::f2 c(kFourPi);
    return c;
}
// scalar read in binary64 (double-float: the integer split, no FP64 unit work)
template <typename PR> __device__ __forceinline__ typename KT<PR>::R scal(typename KT<PR>::T x) { return x; }
template <> __device__ __forceinline__ ff::f2 scal<DD>(double x) { return ff::split_int(x); }

// Per-thread accumulator of the field kernels' reductions: binary64 for
// double, double-float for DD (the computed type) and for float (AccF: the
// binary32 terms summed in a double-float pair).
template <typename PR> struct AccK { typedef typename KT<PR>::R type; };
template <> struct AccK<float> { typedef AccF type; };

// Block totals of per-thread accumulators (double-float ones are added in
// double-float across the warp and in binary64 across warps).
template <int NQ, typename PR> __device__ __forceinline__ void block_total(typename AccK<PR>::type *acc, double *tot)
{
    if constexpr (is_dd<PR>()) {
        block_sum_f2<NQ>(acc, tot);
    } else if constexpr (std::is_same<PR, float>::value) {
        block_sum<NQ>(acc, tot);
    } else {
        block_sum<NQ, double>(acc, tot);
    }
}

// G vector of the half-spectrum point (ix, iy, kz) in the computed
// precision, from the per-axis reciprocal spacings (no divisions).
template <typename A> struct Gk {
    A gx, gy, gz, g2;  // G with +n/2 on Nyquist planes
    A dx, dy, dz;      // first-derivative multipliers (0 on the own-axis Nyquist plane)
    A w;               // Hermitian weight of the half spectrum (1 on kz = 0, nz/2)
    A ig2;             // triclinic cells: (1/G^2 + 1/G'^2)/2 (see RecipB)
};

template <typename A>
__device__ __forceinline__ Gk<A> gvec(const GridInfo &g, A bx, A by, A bz, int ix, int iy, int kz)
{
    Gk<A> r;
    int kx = ix <= g.nx / 2 ? ix : ix - g.nx;
    int ky = iy <= g.ny / 2 ? iy : iy - g.ny;
    r.gx = A(kx) * bx;
    r.gy = A(ky) * by;
    r.gz = A(kz) * bz;
    r.g2 = r.gx * r.gx + r.gy * r.gy + r.gz * r.gz;
    r.dx = (2 * ix == g.nx) ? A(0) : r.gx;
    r.dy = (2 * iy == g.ny) ? A(0) : r.gy;
    r.dz = (2 * kz == g.nz) ? A(0) : r.gz;
    r.w = (kz == 0 || 2 * kz == g.nz) ? A(1) : A(2);
    return r;
}

// First-derivative multiplier along one axis: k b with k the signed index
// of i on an axis of n points, 0 on the Nyquist plane (as Gk's dx, dy, dz).
template <typename A> __device__ __forceinline__ A dmul(int i, int n, A b)
{
    const int k = i <= n / 2 ? i : i - n;
    return (2 * i == n) ? A(0) : A(k) * b;
}

// Reciprocal basis of the x passes in the computed precision.  Orthorhombic
// (TRI = false): per-axis spacings, G_a = k_a b_a.  General cell (TRI =
// true): G = kx b_0 + ky b_1 + kz b_2 (+n/2 on Nyquist planes), and the
// Cartesian first-derivative multiplier D_a = sum_j kd_j (b_j)_a with each
// integer kd_j zeroed on its own Nyquist plane (so gradient and divergence
// stay exact adjoints).  gk: G^2 and Hermitian weight; d: D_a.  In a
// triclinic cell the Nyquist partner G' of a point (its integer indices
// negated except those on their Nyquist plane) is not -G, so |G'| != |G|
// there: even kernels enter as the Hermitian part of the full-box spectrum,
// 1/G^2 -> (1/G^2 + 1/G'^2)/2 (gk's ig2), which is what the real part of
// the full-box inverse transform gives.
template <typename PR, bool TRI> struct RecipB;
template <typename PR> struct RecipB<PR, false> {
    typedef typename KT<PR>::R R;
    R bx, by, bz;
    __device__ __forceinline__ explicit RecipB(const GridInfo &g)
        : bx(gcst<PR>(g.bx, g.bxf, g.bx2)), by(gcst<PR>(g.by, g.byf, g.by2)), bz(gcst<PR>(g.bz, g.bzf, g.bz2))
    {
    }
    __device__ __forceinline__ Gk<R> gk(const GridInfo &g, int ix, int iy, int kz) const
    {
        return gvec<R>(g, bx, by, bz, ix, iy, kz);
    }
    __device__ __forceinline__ R d(const GridInfo &g, int a, int ix, int iy, int kz) const
    {
        return a == 0 ? dmul<R>(ix, g.nx, bx) : (a == 1 ? dmul<R>(iy, g.ny, by) : dmul<R>(kz, g.nz, bz));
    }
};
template <typename PR> struct RecipB<PR, true> {
    typedef typename KT<PR>::R R;
    R b[9];
    __device__ __forceinline__ explicit RecipB(const GridInfo &g)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k) b[k] = gcst<PR>(g.Bm[k], g.Bmf[k], g.Bm2[k]);
    }
    __device__ __forceinline__ Gk<R> gk(const GridInfo &g, int ix, int iy, int kz) const
    {
        Gk<R> r;
        const R kx = R(ix <= g.nx / 2 ? ix : ix - g.nx), ky = R(iy <= g.ny / 2 ? iy : iy - g.ny), kzr = R(kz);
        r.gx = kx * b[0] + ky * b[3] + kzr * b[6];
        r.gy = kx * b[1] + ky * b[4] + kzr * b[7];
        r.gz = kx * b[2] + ky * b[5] + kzr * b[8];
        r.g2 = r.gx * r.gx + r.gy * r.gy + r.gz * r.gz;
        const R px = (2 * ix == g.nx) ? kx : R(0) - kx, py = (2 * iy == g.ny) ? ky : R(0) - ky,
                pz = (2 * kz == g.nz) ? kzr : R(0) - kzr;
        const R qx = px * b[0] + py * b[3] + pz * b[6];
        const R qy = px * b[1] + py * b[4] + pz * b[7];
        const R qz = px * b[2] + py * b[5] + pz * b[8];
        const R g2p = qx * qx + qy * qy + qz * qz;
        r.ig2 = r.g2 > R(0) ? (R(1) / r.g2 + R(1) / g2p) * R(0.5) : R(0);
        r.dx = r.dy = r.dz = R(0);
        r.w = (kz == 0 || 2 * kz == g.nz) ? R(1) : R(2);
        return r;
    }
    __device__ __forceinline__ R d(const GridInfo &g, int a, int ix, int iy, int kz) const
    {
        const int kx = (2 * ix == g.nx) ? 0 : (ix <= g.nx / 2 ? ix : ix - g.nx);
        const int ky = (2 * iy == g.ny) ? 0 : (iy <= g.ny / 2 ? iy : iy - g.ny);
        const int kd = (2 * kz == g.nz) ? 0 : kz;
        return R(kx) * b[a] + R(ky) * b[3 + a] + R(kd) * b[6 + a];
    }
};

// The binary64 routine for points outside the double-float domain, out of
// line so that its registers do not count against the common path.
__device__ __noinline__ PwF2 pw_dd_fallback(const FuncParams &fp, const double *__restrict__ tab, double temp,
                                            ff::f2 n, const ff::f2 *gr, int xc)
{
    PwF2 o;
    const double nd = ff::to_double(n);
    const double gd[3] = {ff::to_double(gr[0]), ff::to_double(gr[1]), ff::to_double(gr[2])};
    PwOut<double> b = pw_point_native<double>(fp, tab, temp, nd, gd[0] * gd[0] + gd[1] * gd[1] + gd[2] * gd[2], xc);
    o.f = ff::f2(b.f);
    o.ts = ff::f2(b.ts);
    o.dfdn = ff::f2(b.dfdn);
    o.eps = ff::f2(b.eps);
    o.vxc = ff::f2(b.vxc);
    for (int a = 0; a < 3; ++a) o.w[a] = ff::f2(b.wc * gd[a]);
    return o;
}

// Pointwise functional of the double-float kernels: the double-float
// routine, and binary64 outside its domain.  n and gr[3] in double-float.
__device__ __forceinline__ PwF2 pw_dd(const FuncParams &fp, const double *__restrict__ tab, ff::f2 tcoef,
                                      double temp, ff::f2 n, const ff::f2 *gr, int xc)
{
    PwF2 o;
    if (pw_core_f2(fp, reinterpret_cast<const ff::f2 *>(tab + kTfSize), tcoef, n, gr, xc, o)) return o;
    return pw_dd_fallback(fp, tab, temp, n, gr, xc);
}

// (row, column) of the element indices threadIdx.x, threadIdx.x +
// blockDim.x, ... in rows of width w, stepped without a division.
struct RowCol {
    int r, c, dr, dc, w;
    __device__ __forceinline__ explicit RowCol(int w_) : w(w_)
    {
        r = threadIdx.x / w_;
        c = threadIdx.x - r * w_;
        dr = blockDim.x / w_;
        dc = blockDim.x - dr * w_;
    }
    __device__ __forceinline__ void next()
    {
        r += dr;
        c += dc;
        if (c >= w) {
            c -= w;
            ++r;
        }
    }
};

// Multiply element e of a line of n by i kt(e) s (kt = 0 on the Nyquist plane).
template <typename CC, typename R>
__device__ __forceinline__ CC times_ik(CC x, int e, int n, R s)
{
    const int k = (2 * e == n) ? 0 : (e <= n / 2 ? e : e - n);
    const R m = R(k) * s;
    return cmk<CC>(R(0) - m * x.y, m * x.x);
}

// Blocks per SM the transform kernels' registers are sized for (launch
// bounds with 256 threads; 0: no bound).
#ifndef OFDFT_FFT_MINB
#define OFDFT_FFT_MINB 4
#endif
#if OFDFT_FFT_MINB > 0
#define OFDFT_FFT_BOUNDS __launch_bounds__(256, OFDFT_FFT_MINB)
#else
#define OFDFT_FFT_BOUNDS
#endif

// ------------------------------------------------------------------ z pass
// Pair p of a block holds real lines 2p (real part) and 2p+1 (imaginary part).

// With dzout the kernel also writes d_z n (the derivative along z by the
// line transforms it already holds: the forward spectrum times i kt ds_z,
// transformed back).
template <typename PR, int MODE>
__global__ void OFDFT_FFT_BOUNDS k_zfwd(GridInfo g, FftAxis az, int P, const typename KT<PR>::T *__restrict__ in,
                       const typename KT<PR>::T *__restrict__ phi, const typename KT<PR>::T *__restrict__ dhat,
                       typename KT<PR>::T c, typename KT<PR>::T s, const void *__restrict__ cs,
                       typename KT<PR>::T *__restrict__ phit, typename KT<PR>::C *__restrict__ out,
                       typename KT<PR>::T *__restrict__ dzout)
{
    typedef typename KT<PR>::T T;
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    if (MODE == 2 && cs != nullptr) {   // rotation angle (two T) from the device CG state
        c = reinterpret_cast<const T *>(cs)[0];
        s = reinterpret_cast<const T *>(cs)[1];
    }
    const R cr = scal<PR>(c), sr = scal<PR>(s);
    extern __shared__ __align__(16) unsigned char smraw[];
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + P * g.nz;
    const long long npairs = (long long)g.nx * g.ny / 2;
    const long long p0 = (long long)blockIdx.x * P;
    const int nl = (int)min((long long)P, npairs - p0);
    const int nz = g.nz, K = g.K;
    const long long base = 2 * p0 * nz;
    RowCol rc(nz);
    for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x, rc.next()) {
        const int line = rc.r, e = rc.c;
        R val;
        if (MODE == 0) {
            val = ldr<PR>(in[base + i]);
        } else if (MODE == 1) {
            R ph = ldr<PR>(phi[base + i]);
            val = ph * ph;
        } else {
            R ph = cr * ldr<PR>(phi[base + i]) + sr * ldr<PR>(dhat[base + i]);
            phit[base + i] = str<PR>(ph);
            val = ph * ph;
        }
        R *dstp = reinterpret_cast<R *>(&A[(line >> 1) * nz + e]);
        dstp[line & 1] = val;
    }
    __syncthreads();
    CC *X = fft_lines<CC, false>(A, B, az, nl, nz, 1, false);
    const long long obase = 2 * p0 * K;
    constexpr R half(0.5), mhalf(-0.5);
    RowCol rk(K);
    for (int i = threadIdx.x; i < 2 * nl * K; i += blockDim.x, rk.next()) {
        const int line = rk.r, k = rk.c;
        const CC *row = X + (line >> 1) * nz;
        CC z = row[k], zc = cconj(row[k == 0 ? 0 : nz - k]);
        CC r = (line & 1) ? cmk<CC>(half * (z.y - zc.y), mhalf * (z.x - zc.x))
                          : cmk<CC>(half * (z.x + zc.x), half * (z.y + zc.y));
        out[obase + i] = stc<PR>(r);
    }
    if (dzout != nullptr) {
        __syncthreads();
        const R sz = gcst<PR>(g.ds[2], g.dsf[2], g.ds2[2]);
        RowCol re(nz);
        for (int i = threadIdx.x; i < nl * nz; i += blockDim.x, re.next())
            X[i] = times_ik<CC, R>(X[i], re.c, nz, sz);
        __syncthreads();
        CC *Y = fft_lines<CC, true>(X, X == A ? B : A, az, nl, nz, 1, false);
        RowCol ro(nz);
        for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x, ro.next()) {
            const R *src = reinterpret_cast<const R *>(&Y[(ro.r >> 1) * nz + ro.c]);
            dzout[base + i] = str<PR>(src[ro.r & 1]);
        }
    }
}

// Build the pair-packed complex line C_k = A_k + i B_k (k <= nz/2) and its
// Hermitian completion C_{nz-k} = conj(A_k) + i conj(B_k); the imaginary
// parts of A_0, A_{nz/2} (and B's) are dropped, as a real inverse does.
template <typename PR>
__device__ __forceinline__ void pack_c2r(const typename KT<PR>::C *__restrict__ src, long long obase, int nl,
                                         int nz, int K, typename KT<PR>::CC *dst)
{
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    RowCol rc(K);
    for (int i = threadIdx.x; i < nl * K; i += blockDim.x, rc.next()) {
        const int p = rc.r, k = rc.c;
        CC a = ldc<PR>(src[obase + (2 * p) * (long long)K + k]);
        CC b = ldc<PR>(src[obase + (2 * p + 1) * (long long)K + k]);
        if (k == 0 || 2 * k == nz) {
            a.y = R(0);
            b.y = R(0);
        }
        dst[p * nz + k] = cmk<CC>(a.x - b.y, a.y + b.x);
        if (k != 0 && 2 * k != nz) dst[p * nz + nz - k] = cmk<CC>(a.x + b.y, b.x - a.y);
    }
}

// Unpack a forward-transformed pair-packed line into two half spectra.
template <typename PR>
__device__ __forceinline__ void unpack_r2c(const typename KT<PR>::CC *X, long long obase, int nl, int nz, int K,
                                           typename KT<PR>::C *__restrict__ out)
{
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    constexpr R half(0.5), mhalf(-0.5);
    RowCol rc(K);
    for (int i = threadIdx.x; i < 2 * nl * K; i += blockDim.x, rc.next()) {
        const int line = rc.r, k = rc.c;
        const CC *row = X + (line >> 1) * nz;
        CC z = row[k], zc = cconj(row[k == 0 ? 0 : nz - k]);
        out[obase + i] = stc<PR>((line & 1) ? cmk<CC>(half * (z.y - zc.y), mhalf * (z.x - zc.x))
                                            : cmk<CC>(half * (z.x + zc.x), half * (z.y + zc.y)));
    }
}

// Final stage: C2R of D(G); v = D(r) + v_part (GGA) or, for ftTF, the
// pointwise functional is evaluated here and added.  Partials (ftTF only
// for the first six): F_s, TS, F_xc, sum(n df/dn - f), 0, sum n(v_xc - eps),
// then sum phi^2 v, sum phi^2, sum 2 phi v dphi/dtheta.
template <typename PR, bool FTTF>
__global__ void k_zfinal(GridInfo g, FftAxis az, int P, const typename KT<PR>::C *__restrict__ dspec,
                         const typename KT<PR>::T *__restrict__ vpart, const typename KT<PR>::T *__restrict__ phit,
                         const typename KT<PR>::T *__restrict__ phi, const typename KT<PR>::T *__restrict__ dhat,
                         typename KT<PR>::T c, typename KT<PR>::T s, const void *__restrict__ cs,
                         typename KT<PR>::T temp, FuncParams fp, const typename KT<PR>::T *__restrict__ tab, int xc,
                         typename KT<PR>::T *__restrict__ vout, double *__restrict__ part)
{
    typedef typename KT<PR>::T T;
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    if (cs != nullptr) {
        c = reinterpret_cast<const T *>(cs)[0];
        s = reinterpret_cast<const T *>(cs)[1];
    }
    const R cr = scal<PR>(c), sr = scal<PR>(s);
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nz = g.nz, K = g.K;
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + P * nz;
    const long long npairs = (long long)g.nx * g.ny / 2;
    const long long p0 = (long long)blockIdx.x * P;
    const int nl = (int)min((long long)P, npairs - p0);
    const long long obase = 2 * p0 * K;
    const long long rbase = 2 * p0 * nz;
    pack_c2r<PR>(dspec, obase, nl, nz, K, A);
    __syncthreads();
    CC *X = fft_lines<CC, true>(A, B, az, nl, nz, 1, false);
    typedef typename AccK<PR>::type AC;
    AC acc[9] = {AC(0), AC(0), AC(0), AC(0), AC(0), AC(0), AC(0), AC(0), AC(0)};
    const ff::f2 tcoef = is_dd<PR>() && FTTF ? ff::f2(2.0 / OF_K23 * (double)temp) : ff::f2(0.0f, 0.0f);
    RowCol rc(nz);
    for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x, rc.next()) {
        const int line = rc.r, e = rc.c;
        CC d = X[(line >> 1) * nz + e];
        R dr = (line & 1) ? d.y : d.x;
        R ph = ldr<PR>(phit[rbase + i]);
        R n = ph * ph;
        R v;
        if (FTTF) {
            R f, ts, dfdn, eps, vxc;
            if constexpr (is_dd<PR>()) {
                const R gz[3] = {R(0), R(0), R(0)};
                const PwF2 o = pw_dd(fp, tab, tcoef, (double)temp, n, gz, xc);
                f = o.f, ts = o.ts, dfdn = o.dfdn, eps = o.eps, vxc = o.vxc;
            } else {
                PwOut<T> o = pw_point_native<T>(fp, tab, temp, n, T(0), xc);
                f = o.f, ts = o.ts, dfdn = o.dfdn, eps = o.eps, vxc = o.vxc;
            }
            v = dfdn + vxc + dr;
            acc[0] += f;
            acc[1] += ts;
            acc[2] += n * eps;
            acc[3] += n * dfdn - f;
            acc[5] += n * (vxc - eps);
        } else {
            v = ldr<PR>(vpart[rbase + i]) + dr;
        }
        vout[rbase + i] = str<PR>(v);
        acc[6] += n * v;
        acc[7] += n;
        if (dhat != nullptr) {
            R dphi = -sr * ldr<PR>(phi[rbase + i]) + cr * ldr<PR>(dhat[rbase + i]);
            acc[8] += R(2) * (ph * v) * dphi;
        }
    }
    double tot[9];
    block_total<9, PR>(acc, tot);
    if (threadIdx.x == 0)
        for (int q = 0; q < 9; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = tot[q];
}

// ------------------------------------------------------------- y/x passes
// Tile: g.tk consecutive columns of the flattened (ix, kz) index space (y
// pass, rows iy) or (iy, kz) space (x pass, rows ix), so every tile but the
// last is full although kz runs over K = nz/2 + 1 values; rows are the
// transformed axis.  Each column's base offset, outer index (ix or iy) and
// kz are worked out once per block into shared memory (columns past the end
// repeat the last one).

struct ColTile {
    long long rstride;
    int ncol, tk, tsh;                // tk = 2^tsh columns (4, 8 or 16)
    const long long *cbase;           // offset of (row 0, column c)
    const int *couter, *ckz;          // ix (y pass) or iy (x pass), and kz
};

__device__ __forceinline__ ColTile col_tile(const GridInfo &g, bool xaxis)
{
    __shared__ long long s_cb[16];
    __shared__ int s_co[16], s_ck[16];
    const int tk = g.tk;
    const long long total = (long long)(xaxis ? g.ny : g.nx) * g.K;
    const long long col0 = (long long)blockIdx.x * tk;
    ColTile t;
    t.tk = tk;
    t.tsh = __ffs(tk) - 1;
    t.ncol = (int)min((long long)tk, total - col0);
    t.rstride = xaxis ? (long long)g.ny * g.K : (long long)g.K;
    if (threadIdx.x < tk) {
        const long long col = col0 + min((int)threadIdx.x, t.ncol - 1);
        const int outer = (int)(col / g.K), kz = (int)(col - (long long)outer * g.K);
        s_co[threadIdx.x] = outer;
        s_ck[threadIdx.x] = kz;
        s_cb[threadIdx.x] = xaxis ? col : (long long)outer * g.ny * g.K + kz;
    }
    __syncthreads();
    t.cbase = s_cb;
    t.couter = s_co;
    t.ckz = s_ck;
    return t;
}

// Column tiles of one field: the grid's x dimension of the y and x passes.
__host__ __device__ __forceinline__ int tiles_of(const GridInfo &g, bool xaxis)
{
    const long long total = (long long)(xaxis ? g.ny : g.nx) * g.K;
    return (int)((total + g.tk - 1) / g.tk);
}

template <typename PR>
__device__ __forceinline__ void load_tile(const typename KT<PR>::C *__restrict__ src, const ColTile &t, int nrows,
                                          typename KT<PR>::CC *dst)
{
    for (int i = threadIdx.x; i < nrows * t.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c < t.ncol) dst[i] = ldc<PR>(src[t.cbase[c] + r * t.rstride]);
    }
}

template <typename PR>
__device__ __forceinline__ void store_tile(typename KT<PR>::C *__restrict__ dst, const ColTile &t, int nrows,
                                           const typename KT<PR>::CC *src)
{
    for (int i = threadIdx.x; i < nrows * t.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c < t.ncol) dst[t.cbase[c] + r * t.rstride] = stc<PR>(src[i]);
    }
}

template <typename PR, bool INV>
__global__ void OFDFT_FFT_BOUNDS k_ypass(GridInfo g, FftAxis ay, typename KT<PR>::C *__restrict__ data, long long fstride)
{
    typedef typename KT<PR>::C C;
    typedef typename KT<PR>::CC CC;
    extern __shared__ __align__(16) unsigned char smraw[];
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + g.ny * g.tk;
    ColTile t = col_tile(g, false);
    C *f = data + blockIdx.y * fstride;
    load_tile<PR>(f, t, g.ny, A);
    __syncthreads();
    CC *X = fft_lines<CC, INV>(A, B, ay, t.ncol, 1, g.tk, true);
    store_tile<PR>(f, t, g.ny, X);
}

// One G-point's share of the LPP pressure (Eq. (pressure), LPP term, at
// fixed Omega n(G) and fractional coordinates).  Gaussian ion: 3x the share,
// Re(n* v_ext)(1 - G^2 rc^2/2) (the caller divides by 3); Heine-Abarenkov
// (Eq. (E4A)) and any form in a triclinic cell: Re(n* v_p) with the
// pressure weights v_p stored after v_ext.
template <typename PR>
__device__ __forceinline__ typename KT<PR>::R ploc_term(const GridInfo &g, const typename KT<PR>::C *vext,
                                                      long long vi, const typename KT<PR>::CC &nG,
                                                      typename KT<PR>::R re, typename KT<PR>::R hr,
                                                      typename KT<PR>::R g2)
{
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    if (g.lpp || g.tri) {
        CC vp = ldc<PR>(vext[g.NH + vi]);
        return nG.x * vp.x + nG.y * vp.y;
    }
    return re * (R(1) - hr * g2);
}

// x pass, ftTF variant: forward x -> energies -> v_HL(G) = 4 pi n/G^2 + v_ext
// inverse-x, written over the spectrum.  If keep_n, n(G) is also stored in nG_out.
template <typename PR, bool TRI>
__global__ void OFDFT_FFT_BOUNDS k_xhl(GridInfo g, FftAxis ax, typename KT<PR>::C *__restrict__ spec,
                      const typename KT<PR>::C *__restrict__ vext, typename KT<PR>::C *__restrict__ nG_out,
                      int inverse, double *__restrict__ part)
{
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx;
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + nx * g.tk;
    ColTile t = col_tile(g, true);
    load_tile<PR>(spec, t, nx, A);
    __syncthreads();
    CC *X = fft_lines<CC, false>(A, B, ax, t.ncol, 1, g.tk, true);
    const RecipB<PR, TRI> rb(g);
    const R hr = gcst<PR>(g.hr, g.hrf, g.hr2);
    const R fpi = fourpi<PR>();
    const R invN = gcst<PR>(g.invN, g.invNf, g.invN2);
    typedef typename AccK<PR>::type AC;
    AC acc[3] = {AC(0), AC(0), AC(0)};
    for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c >= t.ncol) continue;
        CC nG = cscale(X[i], invN);
        Gk<R> k = rb.gk(g, r, t.couter[c], t.ckz[c]);
        const long long vi = t.cbase[c] + r * t.rstride;
        CC ve = ldc<PR>(vext[vi]);
        CC out = cmk<CC>(R(0), R(0));
        if (k.g2 > R(0)) {
            R n2 = nG.x * nG.x + nG.y * nG.y;
            R re = nG.x * ve.x + nG.y * ve.y;
            if constexpr (TRI) acc[0] += k.w * n2 * k.ig2;
            else acc[0] += k.w * n2 / k.g2;
            acc[1] += k.w * re;
            acc[2] += k.w * ploc_term<PR>(g, vext, vi, nG, re, hr, k.g2);
            R kh;
            if constexpr (TRI) kh = fpi * k.ig2;
            else kh = fpi / k.g2;
            out = cmk<CC>(kh * nG.x + ve.x, kh * nG.y + ve.y);
        }
        if (nG_out != nullptr) nG_out[t.cbase[c] + r * t.rstride] = stc<PR>(nG);
        X[i] = out;
    }
    __syncthreads();
    if (inverse) {
        CC *other = (X == A) ? B : A;
        CC *Y = fft_lines<CC, true>(X, other, ax, t.ncol, 1, g.tk, true);
        store_tile<PR>(spec, t, nx, Y);
    }
    double tot[3];
    block_total<3, PR>(acc, tot);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = 0.5 * g.omega * 12.566370614359172954 * tot[0];
        part[(size_t)gridDim.x + blockIdx.x] = g.omega * tot[1];
        part[(size_t)2 * gridDim.x + blockIdx.x] = ((g.lpp || g.tri) ? 1.0 : 1.0 / 3.0) * tot[2];
    }
}

// ------------------------------------------------- derivative line passes
// A GGA evaluation takes the gradient of n and the divergence of W one grid
// axis at a time.  The 3-D transform is a product of commuting 1-D
// transforms and the derivative multiplier along lattice direction j, kt_j
// (the signed integer index, zeroed on its own Nyquist plane), depends on
// k_j alone, so F^-1 (i kt_j) F f = F_j^-1 (i kt_j) F_j f: each derivative
// needs transforms along its own axis only.  The pass multiplies by
// i kt_j ds_j, ds_j = b_j / n_j in an orthorhombic cell (the Cartesian
// derivative) or 1 / n_j in a general cell (the lattice-direction
// derivative; the pointwise kernel combines the three with the reciprocal
// basis, D_a = sum_j kt_j (b_j)_a as in the x passes).  Two real columns
// travel as one complex line c = a + i b: the operator maps real fields to
// real fields, so F^-1 M F c = (d a) + i (d b) needs no unpacking.

// Pair-column tile of a real field for the passes along x (AX 0) or y
// (AX 1): g.dk consecutive pairs of adjacent iz columns of the flattened
// (iy, iz) (x pass) or (ix, iz) (y pass) space; rows run along the axis.
struct PairTile {
    long long rstride;
    int ncol, tk, tsh;
    const long long *cbase;   // offset of (row 0, even column of pair c)
};

__device__ __forceinline__ PairTile pair_tile(const GridInfo &g, int ax)
{
    __shared__ long long s_pb[16];
    const int tk = g.dk;
    const int hz = g.nz / 2;
    const long long total = (long long)(ax == 0 ? g.ny : g.nx) * hz;
    const long long p0 = (long long)blockIdx.x * tk;
    PairTile t;
    t.tk = tk;
    t.tsh = __ffs(tk) - 1;
    t.ncol = (int)min((long long)tk, total - p0);
    t.rstride = ax == 0 ? (long long)g.ny * g.nz : (long long)g.nz;
    if (threadIdx.x < tk) {
        const long long p = p0 + min((int)threadIdx.x, t.ncol - 1);
        long long b = 2 * p;   // x pass: pairs of the yz plane are contiguous
        if (ax == 1) {
            const long long ix = p / hz;
            b = ix * g.ny * g.nz + 2 * (p - ix * hz);
        }
        s_pb[threadIdx.x] = b;
    }
    __syncthreads();
    t.cbase = s_pb;
    return t;
}

__host__ __device__ __forceinline__ int pair_tiles_of(const GridInfo &g, int ax)
{
    const long long total = (long long)(ax == 0 ? g.ny : g.nx) * (g.nz / 2);
    return (int)((total + g.dk - 1) / g.dk);
}

// Stored pair of reals (two adjacent iz columns; even offset, so aligned).
template <typename T> struct Pair2;
template <> struct Pair2<double> { typedef double2 type; };
template <> struct Pair2<float> { typedef float2 type; };

// out (= or +=) d_j f along grid axis AX for f = phi^2 (MODE 0) or f = in
// (MODE 1); ACC 1 adds to out.  out may be in (each block reads its columns
// whole before it writes them, and no other block touches them).
template <typename PR, int AX, int MODE, int ACC>
__global__ void OFDFT_FFT_BOUNDS k_dline(GridInfo g, FftAxis fa, const typename KT<PR>::T *in,
                        typename KT<PR>::T *out)
{
    typedef typename KT<PR>::T T;
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    typedef typename Pair2<T>::type T2;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = AX == 0 ? g.nx : g.ny;
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + n * g.dk;
    const PairTile t = pair_tile(g, AX);
    for (int i = threadIdx.x; i < n * t.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c < t.ncol) {
            const T2 v = *reinterpret_cast<const T2 *>(in + t.cbase[c] + r * t.rstride);
            R a = ldr<PR>(v.x), b = ldr<PR>(v.y);
            if (MODE == 0) {
                a = a * a;
                b = b * b;
            }
            A[i] = cmk<CC>(a, b);
        }
    }
    __syncthreads();
    CC *X = fft_lines<CC, false>(A, B, fa, t.ncol, 1, t.tk, true);
    const R s = gcst<PR>(g.ds[AX], g.dsf[AX], g.ds2[AX]);
    for (int i = threadIdx.x; i < n * t.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c < t.ncol) X[i] = times_ik<CC, R>(X[i], r, n, s);
    }
    __syncthreads();
    CC *Y = fft_lines<CC, true>(X, X == A ? B : A, fa, t.ncol, 1, t.tk, true);
    for (int i = threadIdx.x; i < n * t.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c >= t.ncol) continue;
        T2 *p = reinterpret_cast<T2 *>(out + t.cbase[c] + r * t.rstride);
        const CC y = Y[i];
        T2 o;
        if (ACC) {
            const T2 q = *p;
            o.x = str<PR>(ldr<PR>(q.x) + y.x);
            o.y = str<PR>(ldr<PR>(q.y) + y.y);
        } else {
            o.x = str<PR>(y.x);
            o.y = str<PR>(y.y);
        }
        *p = o;
    }
}

// k_dline with warp-owned lines: the tile is line-major with a padded line
// stride n + 1 (column loads and stores stay coalesced in global memory and
// spread over the shared-memory banks), warp w transforms, multiplies and
// back-transforms lines [w L, (w + 1) L), L = tile width / warps, with
// warp-level synchronisation between stages; the block synchronises only
// after the load and before the store.
template <typename PR, int AX, int MODE, int ACC>
__global__ void OFDFT_FFT_BOUNDS k_dline_ws(GridInfo g, FftAxis fa, const typename KT<PR>::T *in,
                                            typename KT<PR>::T *out)
{
    typedef typename KT<PR>::T T;
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    typedef typename Pair2<T>::type T2;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = AX == 0 ? g.nx : g.ny;
    const int ls = n + 1;
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + ls * g.dk;
    const PairTile t = pair_tile(g, AX);
    for (int i = threadIdx.x; i < n * t.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c < t.ncol) {
            const T2 v = *reinterpret_cast<const T2 *>(in + t.cbase[c] + r * t.rstride);
            R a = ldr<PR>(v.x), b = ldr<PR>(v.y);
            if (MODE == 0) {
                a = a * a;
                b = b * b;
            }
            A[c * ls + r] = cmk<CC>(a, b);
        }
    }
    __syncthreads();
    const int nw = blockDim.x >> 5, lpw = t.tk / nw;
    const int l0 = (threadIdx.x >> 5) * lpw;
    const int nlw = max(0, min(lpw, t.ncol - l0));
    CC *X = fft_lines_w<CC, false>(A, B, fa, l0, nlw, ls);
    const R s = gcst<PR>(g.ds[AX], g.dsf[AX], g.ds2[AX]);
    for (int it = threadIdx.x & 31; it < nlw * n; it += 32) {
        const int m = it / n, r = it - m * n;
        CC *p = X + (l0 + m) * ls + r;
        *p = times_ik<CC, R>(*p, r, n, s);
    }
    __syncwarp();
    CC *Y = fft_lines_w<CC, true>(X, X == A ? B : A, fa, l0, nlw, ls);
    __syncthreads();
    for (int i = threadIdx.x; i < n * t.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c >= t.ncol) continue;
        T2 *p = reinterpret_cast<T2 *>(out + t.cbase[c] + r * t.rstride);
        const CC y = Y[c * ls + r];
        T2 o;
        if (ACC) {
            const T2 q = *p;
            o.x = str<PR>(ldr<PR>(q.x) + y.x);
            o.y = str<PR>(ldr<PR>(q.y) + y.y);
        } else {
            o.x = str<PR>(y.x);
            o.y = str<PR>(y.y);
        }
        *p = o;
    }
}

// ------------------------------------------------------ pointwise stage
// Pointwise functional + XC at every grid point (Eqs. (tred), (FGGA),
// (vftGGA) first two lines, (vxc1)), no transforms: reads phi and the three
// derivatives of n from d0..d2, writes v_part = df/dn + v_xc and, over
// d0..d2, the fields whose derivatives make up div W: U_j = W_j
// (orthorhombic) or U_j = sum_a (b_j)_a W_a (general cell, where d_j are
// lattice-direction derivatives and grad_a n = sum_j (b_j)_a d_j n).
// Partials: F_s, TS, F_xc, sum(n df/dn - f), sum W.grad n,
// sum n(v_xc - eps_xc); with STRESS also sum W_a d_b n for ab = xx, yy,
// zz, xy, xz, yz (the gradient part of Eq. (stressTF_b)) in rows 6..11.
// Threads per block of the pointwise kernel and the blocks per SM its
// register budget is sized for (launch bounds).
#ifndef OFDFT_PW_THREADS
#define OFDFT_PW_THREADS 256
#endif
#ifndef OFDFT_PW_MINB
#define OFDFT_PW_MINB 3
#endif

template <typename PR, bool STRESS, bool TRI>
__global__ void __launch_bounds__(OFDFT_PW_THREADS, OFDFT_PW_MINB) k_pw(GridInfo g, typename KT<PR>::T *__restrict__ d0, typename KT<PR>::T *__restrict__ d1,
                     typename KT<PR>::T *__restrict__ d2, const typename KT<PR>::T *__restrict__ phit,
                     typename KT<PR>::T temp, FuncParams fp, const typename KT<PR>::T *__restrict__ tab, int xc,
                     typename KT<PR>::T *__restrict__ vpart, double *__restrict__ part)
{
    typedef typename KT<PR>::T T;
    typedef typename KT<PR>::R R;
    typedef typename AccK<PR>::type AC;
    AC acc[6] = {AC(0), AC(0), AC(0), AC(0), AC(0), AC(0)};
    AC sacc[STRESS ? 6 : 1];
    if constexpr (STRESS)
        for (int q = 0; q < 6; ++q) sacc[q] = AC(0);
    R bm[TRI ? 9 : 1];
    if constexpr (TRI)
        for (int k = 0; k < 9; ++k) bm[k] = gcst<PR>(g.Bm[k], g.Bmf[k], g.Bm2[k]);
    const ff::f2 tcoef = is_dd<PR>() ? ff::f2(2.0 / OF_K23 * (double)temp) : ff::f2(0.0f, 0.0f);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
         i += (long long)gridDim.x * blockDim.x) {
        const R dj[3] = {ldr<PR>(d0[i]), ldr<PR>(d1[i]), ldr<PR>(d2[i])};
        R gr[3];
        if constexpr (TRI) {
            for (int a = 0; a < 3; ++a) gr[a] = bm[a] * dj[0] + bm[3 + a] * dj[1] + bm[6 + a] * dj[2];
        } else {
            for (int a = 0; a < 3; ++a) gr[a] = dj[a];
        }
        R w[3];
        if constexpr (is_dd<PR>()) {
            const R ph = ldr<PR>(phit[i]);
            const R n = ph * ph;
            const PwF2 o = pw_dd(fp, tab, tcoef, (double)temp, n, gr, xc);
            vpart[i] = str<PR>(o.dfdn + o.vxc);
            acc[0] += o.f;
            acc[1] += o.ts;
            acc[2] += n * o.eps;
            acc[3] += n * o.dfdn - o.f;
            acc[4] += o.w[0] * gr[0] + o.w[1] * gr[1] + o.w[2] * gr[2];
            acc[5] += n * (o.vxc - o.eps);
            for (int a = 0; a < 3; ++a) w[a] = o.w[a];
        } else {
            const T ph = phit[i];
            const T n = ph * ph;
            const T gg = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
            const PwOut<T> o = pw_point_native<T>(fp, tab, temp, n, gg, xc);
            vpart[i] = o.dfdn + o.vxc;
            acc[0] += o.f;
            acc[1] += o.ts;
            acc[2] += n * o.eps;
            acc[3] += n * o.dfdn - o.f;
            acc[4] += o.wc * gg;
            acc[5] += n * (o.vxc - o.eps);
            for (int a = 0; a < 3; ++a) w[a] = o.wc * gr[a];
        }
        if constexpr (STRESS) {
            sacc[0] += w[0] * gr[0];
            sacc[1] += w[1] * gr[1];
            sacc[2] += w[2] * gr[2];
            sacc[3] += w[0] * gr[1];
            sacc[4] += w[0] * gr[2];
            sacc[5] += w[1] * gr[2];
        }
        if constexpr (TRI) {
            d0[i] = str<PR>(bm[0] * w[0] + bm[1] * w[1] + bm[2] * w[2]);
            d1[i] = str<PR>(bm[3] * w[0] + bm[4] * w[1] + bm[5] * w[2]);
            d2[i] = str<PR>(bm[6] * w[0] + bm[7] * w[1] + bm[8] * w[2]);
        } else {
            d0[i] = str<PR>(w[0]);
            d1[i] = str<PR>(w[1]);
            d2[i] = str<PR>(w[2]);
        }
    }
    double tot[6];
    block_total<6, PR>(acc, tot);
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = tot[q];
    if constexpr (STRESS) {
        __syncthreads();
        block_total<6, PR>(sacc, tot);
        if (threadIdx.x == 0)
            for (int q = 0; q < 6; ++q) part[(size_t)(6 + q) * gridDim.x + blockIdx.x] = tot[q];
    }
}

// Final stage of a GGA evaluation: v = v_HL - d_z U_z + v_part - div, with
// v_HL from the half spectrum dspec (Hartree + LPP after the inverse x and
// y passes), d_z U_z from the pair-packed lines of U_z (forward z transform,
// times i kt ds_z, added to the packed spectrum of v_HL, so one inverse
// transform serves both) and div = d_x U_x + d_y U_y, given as one field or
// as two (div + div2; div2 may be null).  div may alias vout (each point is
// read before it is written, by the same thread).  Partials
// (as k_zfinal's GGA form): rows 0..5 zero, then sum phi^2 v, sum phi^2,
// sum 2 phi v dphi/dtheta.
template <typename PR>
__global__ void OFDFT_FFT_BOUNDS k_zfinal_g(GridInfo g, FftAxis az, int P, const typename KT<PR>::C *__restrict__ dspec,
                           const typename KT<PR>::T *__restrict__ uz, const typename KT<PR>::T *__restrict__ vpart,
                           const typename KT<PR>::T *div, const typename KT<PR>::T *__restrict__ div2,
                           const typename KT<PR>::T *__restrict__ phit,
                           const typename KT<PR>::T *__restrict__ phi, const typename KT<PR>::T *__restrict__ dhat,
                           typename KT<PR>::T c, typename KT<PR>::T s, const void *__restrict__ cs,
                           typename KT<PR>::T *vout, double *__restrict__ part)
{
    typedef typename KT<PR>::T T;
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::CC CC;
    typedef typename AccK<PR>::type AC;
    if (cs != nullptr) {
        c = reinterpret_cast<const T *>(cs)[0];
        s = reinterpret_cast<const T *>(cs)[1];
    }
    const R cr = scal<PR>(c), sr = scal<PR>(s);
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nz = g.nz, K = g.K;
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + P * nz;
    CC *D = B + P * nz;
    const long long npairs = (long long)g.nx * g.ny / 2;
    const long long p0 = (long long)blockIdx.x * P;
    const int nl = (int)min((long long)P, npairs - p0);
    const long long obase = 2 * p0 * K;
    const long long rbase = 2 * p0 * nz;
    pack_c2r<PR>(dspec, obase, nl, nz, K, A);
    {
        RowCol rc(nz);
        for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x, rc.next()) {
            R *dst = reinterpret_cast<R *>(&B[(rc.r >> 1) * nz + rc.c]);
            dst[rc.r & 1] = ldr<PR>(uz[rbase + i]);
        }
    }
    __syncthreads();
    CC *Z = fft_lines<CC, false>(B, D, az, nl, nz, 1, false);
    const R sz = gcst<PR>(g.ds[2], g.dsf[2], g.ds2[2]);
    {
        RowCol re(nz);
        for (int i = threadIdx.x; i < nl * nz; i += blockDim.x, re.next()) {
            const CC d = times_ik<CC, R>(Z[i], re.c, nz, sz);
            A[i] = cmk<CC>(A[i].x - d.x, A[i].y - d.y);
        }
    }
    __syncthreads();
    CC *X = fft_lines<CC, true>(A, Z, az, nl, nz, 1, false);
    AC acc[9] = {AC(0), AC(0), AC(0), AC(0), AC(0), AC(0), AC(0), AC(0), AC(0)};
    RowCol rc(nz);
    for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x, rc.next()) {
        const CC d = X[(rc.r >> 1) * nz + rc.c];
        const R dr = (rc.r & 1) ? d.y : d.x;
        const R ph = ldr<PR>(phit[rbase + i]);
        const R n = ph * ph;
        R v = ldr<PR>(vpart[rbase + i]) + dr - ldr<PR>(div[rbase + i]);
        if (div2 != nullptr) v = v - ldr<PR>(div2[rbase + i]);
        vout[rbase + i] = str<PR>(v);
        acc[6] += n * v;
        acc[7] += n;
        if (dhat != nullptr) {
            const R dphi = -sr * ldr<PR>(phi[rbase + i]) + cr * ldr<PR>(dhat[rbase + i]);
            acc[8] += R(2) * (ph * v) * dphi;
        }
    }
    double tot[9];
    block_total<9, PR>(acc, tot);
    if (threadIdx.x == 0)
        for (int q = 0; q < 9; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = tot[q];
}

int zpairs_per_block(const GridInfo &g)
{
    if (g.zP > 0) return g.zP;
    long long npairs = (long long)g.nx * g.ny / 2;
    int P = (int)(npairs / 608);
    if (P > 8) P = 8;
    if (P < 1) P = 1;
    while (P > 1 && (long long)P * g.nz > 2048) --P;
    return P;
}

// zfwd and zfinal do little work per point: at least 4 pairs per block
// (when the tuned z shape has fewer) so their transforms fill the block.
int zpairs_light(const GridInfo &g)
{
    int P = zpairs_per_block(g);
    if (P < 4) P = 4;
    while (P > 1 && (long long)P * g.nz > 2048) --P;
    return P;
}

int threads_for(int work)
{
    int t = 64;
    while (t < 256 && t < work) t *= 2;
    return t;
}

// Launch the double-float kernels when an FP64 grid asks for them.
#define OFDFT_DISPATCH(T, g, CALL)                          \
    do {                                                    \
        if constexpr (std::is_same<T, double>::value) {     \
            if ((g).dd) {                                   \
                CALL(DD);                                   \
                break;                                      \
            }                                               \
        }                                                   \
        CALL(T);                                            \
    } while (0)

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_zfwd(const GridInfo &g, const FftAxis &az, int mode, const T *in, const T *phi,
                 const T *dhat, T c, T s, const void *cs, T *phit, cplx<T> *out, cudaStream_t st, T *dz)
{
    int P = zpairs_light(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 2 * (size_t)P * g.nz * sizeof(cplx<T>);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
#define CALL(PR)                                                                                              \
    if (mode == 0) k_zfwd<PR, 0><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out, dz);     \
    else if (mode == 1) k_zfwd<PR, 1><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out, dz); \
    else k_zfwd<PR, 2><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out, dz)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
}

namespace {
template <typename PR>
void dline_call(const GridInfo &g, const FftAxis &fa, int axis, int mode, int acc, const typename KT<PR>::T *in,
                typename KT<PR>::T *out, int blocks, int th, size_t sm, cudaStream_t st)
{
    if (g.dws && th % 32 == 0 && g.dk % (th / 32) == 0) {   // whole lines for every warp
        if (axis == 0) {
            if (mode == 0) k_dline_ws<PR, 0, 0, 0><<<blocks, th, sm, st>>>(g, fa, in, out);
            else if (acc == 0) k_dline_ws<PR, 0, 1, 0><<<blocks, th, sm, st>>>(g, fa, in, out);
            else k_dline_ws<PR, 0, 1, 1><<<blocks, th, sm, st>>>(g, fa, in, out);
        } else {
            if (mode == 0) k_dline_ws<PR, 1, 0, 0><<<blocks, th, sm, st>>>(g, fa, in, out);
            else if (acc == 0) k_dline_ws<PR, 1, 1, 0><<<blocks, th, sm, st>>>(g, fa, in, out);
            else k_dline_ws<PR, 1, 1, 1><<<blocks, th, sm, st>>>(g, fa, in, out);
        }
        return;
    }
    if (axis == 0) {
        if (mode == 0) k_dline<PR, 0, 0, 0><<<blocks, th, sm, st>>>(g, fa, in, out);
        else if (acc == 0) k_dline<PR, 0, 1, 0><<<blocks, th, sm, st>>>(g, fa, in, out);
        else k_dline<PR, 0, 1, 1><<<blocks, th, sm, st>>>(g, fa, in, out);
    } else {
        if (mode == 0) k_dline<PR, 1, 0, 0><<<blocks, th, sm, st>>>(g, fa, in, out);
        else if (acc == 0) k_dline<PR, 1, 1, 0><<<blocks, th, sm, st>>>(g, fa, in, out);
        else k_dline<PR, 1, 1, 1><<<blocks, th, sm, st>>>(g, fa, in, out);
    }
}
}  // namespace

template <typename T>
void launch_dline(const GridInfo &g, const FftAxis &fa, int axis, int mode, int acc, const T *in, T *out,
                  cudaStream_t st)
{
    const int n = axis == 0 ? g.nx : g.ny;
    const int blocks = pair_tiles_of(g, axis);
    const size_t sm = 2 * (size_t)(g.dws ? n + 1 : n) * g.dk * sizeof(cplx<T>);
    const int th = g.dth > 0 ? g.dth : threads_for(n * g.dk / 2);   // warp-owned lines: dk a multiple of th / 32
#define CALL(PR) dline_call<PR>(g, fa, axis, mode, acc, in, out, blocks, th, sm, st)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
}

// Blocks of the pointwise kernel: about eight points a thread (the block
// sums cost a few hundred instructions a thread), at least one full wave of
// the GPU's SMs, at most one block per z line pair (the partial-sum rows
// hold nx ny / 2 columns).
int pw_blocks(const GridInfo &g, int th)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            sms = n;
        else
            sms = 152;
    }
    const long long npairs = (long long)g.nx * g.ny / 2;
    long long b = (g.N + 8LL * th - 1) / (8LL * th);
    b = std::max<long long>(b, (long long)sms * OFDFT_PW_MINB);
    b = std::min<long long>(b, (g.N + th - 1) / th);
    return (int)std::min<long long>(b, npairs);
}

template <typename T>
int launch_pw(const GridInfo &g, T *d0, T *d1, T *d2, const T *phit, T temp, const FuncParams &fp, const T *tab,
              int xc, T *vpart, double *part, bool stress, cudaStream_t st)
{
    const int th = OFDFT_PW_THREADS;
    const int blocks = pw_blocks(g, th);
#define CALL(PR)                                                                                              \
    if (stress) {                                                                                             \
        if constexpr (!std::is_same<PR, float>::value) {                                                      \
            if (g.tri) k_pw<PR, true, true><<<blocks, th, 0, st>>>(g, d0, d1, d2, phit, temp, fp, tab, xc, vpart, part); \
            else k_pw<PR, true, false><<<blocks, th, 0, st>>>(g, d0, d1, d2, phit, temp, fp, tab, xc, vpart, part);     \
        }                                                                                                     \
    } else if (g.tri) {                                                                                       \
        k_pw<PR, false, true><<<blocks, th, 0, st>>>(g, d0, d1, d2, phit, temp, fp, tab, xc, vpart, part);    \
    } else {                                                                                                  \
        k_pw<PR, false, false><<<blocks, th, 0, st>>>(g, d0, d1, d2, phit, temp, fp, tab, xc, vpart, part);   \
    }
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
    return blocks;
}

template <typename T>
int launch_zfinal(const GridInfo &g, const FftAxis &az, bool fttf, const cplx<T> *dspec,
                  const T *vpart, const T *phit, const T *phi, const T *dhat, T c, T s,
                  const void *cs, T temp, const FuncParams &fp, const T *tab, int xc, T *vout,
                  double *part, cudaStream_t st)
{
    int P = zpairs_light(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 2 * (size_t)P * g.nz * sizeof(cplx<T>);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
#define CALL(PR)                                                                                       \
    if (fttf)                                                                                          \
        k_zfinal<PR, true><<<blocks, th, sm, st>>>(g, az, P, dspec, vpart, phit, phi, dhat, c, s, cs,  \
                                                   temp, fp, tab, xc, vout, part);                     \
    else                                                                                               \
        k_zfinal<PR, false><<<blocks, th, sm, st>>>(g, az, P, dspec, vpart, phit, phi, dhat, c, s, cs, \
                                                    temp, fp, tab, xc, vout, part)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
    return blocks;
}

template <typename T>
int launch_zfinal_gga(const GridInfo &g, const FftAxis &az, const cplx<T> *dspec, const T *uz, const T *vpart,
                      const T *div, const T *div2, const T *phit, const T *phi, const T *dhat, T c, T s,
                      const void *cs, T *vout, double *part, cudaStream_t st)
{
    int P = zpairs_light(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 3 * (size_t)P * g.nz * sizeof(cplx<T>);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
#define CALL(PR) \
    k_zfinal_g<PR><<<blocks, th, sm, st>>>(g, az, P, dspec, uz, vpart, div, div2, phit, phi, dhat, c, s, cs, vout, \
                                           part)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
    return blocks;
}

template <typename T>
void launch_ypass(const GridInfo &g, const FftAxis &ay, bool inv, cplx<T> *data, int nfields,
                  long long fstride, cudaStream_t st)
{
    dim3 grid(tiles_of(g, false), nfields);
    size_t sm = 2 * (size_t)g.ny * g.tk * sizeof(cplx<T>);
    int th = g.xth > 0 ? g.xth : threads_for(g.ny * g.tk / 2);
#define CALL(PR)                                                            \
    if (inv) k_ypass<PR, true><<<grid, th, sm, st>>>(g, ay, data, fstride); \
    else k_ypass<PR, false><<<grid, th, sm, st>>>(g, ay, data, fstride)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
}

template <typename T>
int launch_xhl(const GridInfo &g, const FftAxis &ax, cplx<T> *spec, const cplx<T> *vext,
               cplx<T> *nG_out, int inverse, double *part, cudaStream_t st)
{
    int blocks = tiles_of(g, true);
    size_t sm = 2 * (size_t)g.nx * g.tk * sizeof(cplx<T>);
    int th = g.xth > 0 ? g.xth : threads_for(g.nx * g.tk / 2);
#define CALL(PR)                                                                             \
    if (g.tri) k_xhl<PR, true><<<blocks, th, sm, st>>>(g, ax, spec, vext, nG_out, inverse, part); \
    else k_xhl<PR, false><<<blocks, th, sm, st>>>(g, ax, spec, vext, nG_out, inverse, part)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
    return blocks;
}

int xpass_blocks(const GridInfo &g) { return tiles_of(g, true); }

int fft_max_threads() { return OFDFT_FFT_MINB > 0 ? 256 : 1024; }

size_t field_smem_max(const GridInfo &g, size_t csize)
{
    int P = zpairs_light(g);
    size_t z = 3 * (size_t)P * g.nz * csize;
    size_t y = 2 * (size_t)g.ny * g.tk * csize;
    size_t x = 2 * (size_t)g.nx * g.tk * csize;
    size_t d = 2 * (size_t)((g.nx > g.ny ? g.nx : g.ny) + (g.dws ? 1 : 0)) * g.dk * csize;
    size_t m = z > y ? z : y;
    m = m > x ? m : x;
    return m > d ? m : d;
}

namespace {
template <typename PR> cudaError_t smem_limits(int b)
{
    cudaError_t e[] = {
        cudaFuncSetAttribute(k_zfwd<PR, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfwd<PR, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfwd<PR, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfinal<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfinal<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfinal_g<PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_ypass<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_ypass<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xhl<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xhl<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline<PR, 0, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline<PR, 0, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline<PR, 0, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline<PR, 1, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline<PR, 1, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline<PR, 1, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline_ws<PR, 0, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline_ws<PR, 0, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline_ws<PR, 0, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline_ws<PR, 1, 0, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline_ws<PR, 1, 1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_dline_ws<PR, 1, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}
}  // namespace

template <typename T> cudaError_t set_field_smem_limits(size_t bytes)
{
    cudaError_t e = smem_limits<T>((int)bytes);
    if (e == cudaSuccess && std::is_same<T, double>::value) e = smem_limits<DD>((int)bytes);
    return e;
}

#define OFDFT_INST(T)                                                                              \
    template void launch_zfwd<T>(const GridInfo &, const FftAxis &, int, const T *, const T *,     \
                                 const T *, T, T, const void *, T *, cplx<T> *, cudaStream_t, T *); \
    template void launch_dline<T>(const GridInfo &, const FftAxis &, int, int, int, const T *, T *, \
                                  cudaStream_t);                                                  \
    template int launch_pw<T>(const GridInfo &, T *, T *, T *, const T *, T, const FuncParams &,   \
                              const T *, int, T *, double *, bool, cudaStream_t);                 \
    template int launch_zfinal<T>(const GridInfo &, const FftAxis &, bool, const cplx<T> *,        \
                                  const T *, const T *, const T *, const T *, T, T, const void *,   \
                                  T, const FuncParams &, const T *, int, T *, double *,            \
                                  cudaStream_t);                                                  \
    template int launch_zfinal_gga<T>(const GridInfo &, const FftAxis &, const cplx<T> *, const T *, \
                                      const T *, const T *, const T *, const T *, const T *,      \
                                      const T *, T, T, const void *, T *, double *, cudaStream_t); \
    template void launch_ypass<T>(const GridInfo &, const FftAxis &, bool, cplx<T> *, int,         \
                                  long long, cudaStream_t);                                       \
    template int launch_xhl<T>(const GridInfo &, const FftAxis &, cplx<T> *, const cplx<T> *,      \
                               cplx<T> *, int, double *, cudaStream_t);                          \
    template cudaError_t set_field_smem_limits<T>(size_t);

OFDFT_INST(double)
OFDFT_INST(float)

}  // namespace ofdft
