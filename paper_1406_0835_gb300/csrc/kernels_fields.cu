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

// Block totals of per-thread accumulators (double-float ones are converted
// to binary64 first; from the warp level up the sums are binary64).
template <int NQ, typename PR> __device__ __forceinline__ void block_total(typename AccK<PR>::type *acc, double *tot)
{
    if constexpr (is_dd<PR>()) {
        double d[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) d[q] = ff::to_double(acc[q]);
        block_sum<NQ, double>(d, tot);
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

// Pointwise functional of the double-float z passes: the double-float
// routine, and binary64 outside its domain.  n and gr[3] in double-float.
__device__ __forceinline__ PwF2 pw_dd(const FuncParams &fp, const double *__restrict__ tab, ff::f2 tcoef,
                                      double temp, ff::f2 n, const ff::f2 *gr, int xc)
{
    PwF2 o;
    if (pw_core_f2(fp, reinterpret_cast<const ff::f2 *>(tab + kTfSize), tcoef, n, gr, xc, o)) return o;
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

// ------------------------------------------------------------------ z pass
// Pair p of a block holds real lines 2p (real part) and 2p+1 (imaginary part).

template <typename PR, int MODE>
__global__ void k_zfwd(GridInfo g, FftAxis az, int P, const typename KT<PR>::T *__restrict__ in,
                       const typename KT<PR>::T *__restrict__ phi, const typename KT<PR>::T *__restrict__ dhat,
                       typename KT<PR>::T c, typename KT<PR>::T s, const void *__restrict__ cs,
                       typename KT<PR>::T *__restrict__ phit, typename KT<PR>::C *__restrict__ out)
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
    const R half = R(0.5), mhalf = R(-0.5);
    RowCol rk(K);
    for (int i = threadIdx.x; i < 2 * nl * K; i += blockDim.x, rk.next()) {
        const int line = rk.r, k = rk.c;
        const CC *row = X + (line >> 1) * nz;
        CC z = row[k], zc = cconj(row[k == 0 ? 0 : nz - k]);
        CC r = (line & 1) ? cmk<CC>(half * (z.y - zc.y), mhalf * (z.x - zc.x))
                          : cmk<CC>(half * (z.x + zc.x), half * (z.y + zc.y));
        out[obase + i] = stc<PR>(r);
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
    const R half = R(0.5), mhalf = R(-0.5);
    RowCol rc(K);
    for (int i = threadIdx.x; i < 2 * nl * K; i += blockDim.x, rc.next()) {
        const int line = rc.r, k = rc.c;
        const CC *row = X + (line >> 1) * nz;
        CC z = row[k], zc = cconj(row[k == 0 ? 0 : nz - k]);
        out[obase + i] = stc<PR>((line & 1) ? cmk<CC>(half * (z.y - zc.y), mhalf * (z.x - zc.x))
                                            : cmk<CC>(half * (z.x + zc.x), half * (z.y + zc.y)));
    }
}

// Fused GGA stage: C2R of grad n (3 fields), pointwise functional + XC,
// R2C of W (3 fields, written over grad n).  Partials: F_s, TS, F_xc,
// sum(n df/dn - f), sum W.grad n, sum n(v_xc - eps_xc); with STRESS also
// sum W_a d_b n for ab = xx, yy, zz, xy, xz, yz (the gradient part of
// Eq. (stressTF_b)) in partial rows 6..11.
template <typename PR, bool STRESS>
__global__ void k_zgga(GridInfo g, FftAxis az, int P, typename KT<PR>::C *__restrict__ g0,
                       typename KT<PR>::C *__restrict__ g1, typename KT<PR>::C *__restrict__ g2,
                       const typename KT<PR>::T *__restrict__ phit, typename KT<PR>::T temp, FuncParams fp,
                       const typename KT<PR>::T *__restrict__ tab, int xc, typename KT<PR>::T *__restrict__ vpart,
                       double *__restrict__ part)
{
    typedef typename KT<PR>::T T;
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::C C;
    typedef typename KT<PR>::CC CC;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nz = g.nz, K = g.K;
    // the three components' lines side by side (field a at line a nl), so
    // each transform is one batch of 3 nl lines; the other half is scratch
    const long long npairs = (long long)g.nx * g.ny / 2;
    const long long p0 = (long long)blockIdx.x * P;
    const int nl = (int)min((long long)P, npairs - p0);
    const long long obase = 2 * p0 * K;
    const long long rbase = 2 * p0 * nz;
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + 3 * P * nz;
    C *spec[3] = {g0, g1, g2};
    for (int a = 0; a < 3; ++a) pack_c2r<PR>(spec[a], obase, nl, nz, K, A + a * nl * nz);
    __syncthreads();
    CC *X = fft_lines<CC, true>(A, B, az, 3 * nl, nz, 1, false);
    CC *res[3] = {X, X + nl * nz, X + 2 * nl * nz};
    typedef typename AccK<PR>::type AC;
    AC acc[6] = {AC(0), AC(0), AC(0), AC(0), AC(0), AC(0)};
    AC sacc[STRESS ? 6 : 1];
    if constexpr (STRESS)
        for (int q = 0; q < 6; ++q) sacc[q] = AC(0);
    const ff::f2 tcoef = is_dd<PR>() ? ff::f2(2.0 / OF_K23 * (double)temp) : ff::f2(0.0f, 0.0f);
    RowCol rc(nz);
    for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x, rc.next()) {
        const int line = rc.r, e = rc.c;
        const int p = line >> 1, hi = line & 1;
        R gr[3];
        for (int a = 0; a < 3; ++a)   // each thread owns one component of the packed pair
            gr[a] = reinterpret_cast<const R *>(&res[a][p * nz + e])[hi];
        if constexpr (is_dd<PR>()) {
            const R ph = ldr<PR>(phit[rbase + i]);
            const R n = ph * ph;
            const PwF2 o = pw_dd(fp, tab, tcoef, (double)temp, n, gr, xc);
            vpart[rbase + i] = str<PR>(o.dfdn + o.vxc);
            acc[0] += o.f;
            acc[1] += o.ts;
            acc[2] += n * o.eps;
            acc[3] += n * o.dfdn - o.f;
            acc[4] += o.w[0] * gr[0] + o.w[1] * gr[1] + o.w[2] * gr[2];
            acc[5] += n * (o.vxc - o.eps);
            if constexpr (STRESS) {
                sacc[0] += o.w[0] * gr[0];
                sacc[1] += o.w[1] * gr[1];
                sacc[2] += o.w[2] * gr[2];
                sacc[3] += o.w[0] * gr[1];
                sacc[4] += o.w[0] * gr[2];
                sacc[5] += o.w[1] * gr[2];
            }
            for (int a = 0; a < 3; ++a) {
                R *d = reinterpret_cast<R *>(&res[a][p * nz + e]);
                d[hi] = o.w[a];
            }
        } else {
            T ph = phit[rbase + i];
            T n = ph * ph;
            T gg = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
            PwOut<T> o = pw_point_native<T>(fp, tab, temp, n, gg, xc);
            const T eps = o.eps, vxc = o.vxc;
            vpart[rbase + i] = o.dfdn + vxc;
            acc[0] += o.f;
            acc[1] += o.ts;
            acc[2] += n * eps;
            acc[3] += n * o.dfdn - o.f;
            acc[4] += o.wc * gg;
            acc[5] += n * (vxc - eps);
            if constexpr (STRESS) {
                sacc[0] += o.wc * gr[0] * gr[0];
                sacc[1] += o.wc * gr[1] * gr[1];
                sacc[2] += o.wc * gr[2] * gr[2];
                sacc[3] += o.wc * gr[0] * gr[1];
                sacc[4] += o.wc * gr[0] * gr[2];
                sacc[5] += o.wc * gr[1] * gr[2];
            }
            for (int a = 0; a < 3; ++a) {
                T *d = reinterpret_cast<T *>(&res[a][p * nz + e]);
                d[hi] = o.wc * gr[a];
            }
        }
    }
    __syncthreads();
    CC *Y = fft_lines<CC, false>(X, X == A ? B : A, az, 3 * nl, nz, 1, false);
    for (int a = 0; a < 3; ++a) unpack_r2c<PR>(Y + a * nl * nz, obase, nl, nz, K, spec[a]);
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
__global__ void k_ypass(GridInfo g, FftAxis ay, typename KT<PR>::C *__restrict__ data, long long fstride)
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

// x pass, gradient variant: forward x -> n(G) (stored), energies, then
// i D_a n(G) inverse-x for a = x, y, z.  Partials: E_H, E_loc, P_loc.
template <typename PR, bool TRI>
__global__ void k_xgrad(GridInfo g, FftAxis ax, typename KT<PR>::C *__restrict__ nspec,
                        const typename KT<PR>::C *__restrict__ vext, typename KT<PR>::C *__restrict__ g0,
                        typename KT<PR>::C *__restrict__ g1, typename KT<PR>::C *__restrict__ g2,
                        double *__restrict__ part)
{
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::C C;
    typedef typename KT<PR>::CC CC;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx;
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + nx * g.tk;
    CC *N = B + nx * g.tk;
    ColTile t = col_tile(g, true);
    load_tile<PR>(nspec, t, nx, A);
    __syncthreads();
    CC *X = fft_lines<CC, false>(A, B, ax, t.ncol, 1, g.tk, true);
    const RecipB<PR, TRI> rb(g);
    const R hr = gcst<PR>(g.hr, g.hrf, g.hr2);
    const R invN = gcst<PR>(g.invN, g.invNf, g.invN2);
    typedef typename AccK<PR>::type AC;
    AC acc[3] = {AC(0), AC(0), AC(0)};   // sum w |n|^2/G^2, sum w Re(n* v_ext), sum w Re(n* v_ext)(1 - G^2 rc^2/2)
    for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c >= t.ncol) continue;
        CC nG = cscale(X[i], invN);
        N[i] = nG;
        Gk<R> k = rb.gk(g, r, t.couter[c], t.ckz[c]);
        if (k.g2 > R(0)) {
            const long long vi = t.cbase[c] + r * t.rstride;
            CC ve = ldc<PR>(vext[vi]);
            R n2 = nG.x * nG.x + nG.y * nG.y;
            R re = nG.x * ve.x + nG.y * ve.y;
            if constexpr (TRI) acc[0] += k.w * n2 * k.ig2;
            else acc[0] += k.w * n2 / k.g2;
            acc[1] += k.w * re;
            acc[2] += k.w * ploc_term<PR>(g, vext, vi, nG, re, hr, k.g2);
        }
    }
    __syncthreads();
    store_tile<PR>(nspec, t, nx, N);
    C *outs[3] = {g0, g1, g2};
    for (int a = 0; a < 3; ++a) {
        for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
            const int r = i >> t.tsh, c = i & (t.tk - 1);
            const R d = rb.d(g, a, r, t.couter[c], t.ckz[c]);
            CC v = N[i];
            A[i] = cmk<CC>(-d * v.y, d * v.x);      // i D_a n(G)
        }
        __syncthreads();
        CC *Y = fft_lines<CC, true>(A, B, ax, t.ncol, 1, g.tk, true);
        store_tile<PR>(outs[a], t, nx, Y);
        __syncthreads();
    }
    double tot[3];
    block_total<3, PR>(acc, tot);
    if (threadIdx.x == 0) {
        // E_H = (Omega/2) sum 4 pi |n|^2/G^2, E_loc = Omega sum Re(n* v_ext),
        // P_loc = sum Re(n* v_p) (ploc_term)
        part[blockIdx.x] = 0.5 * g.omega * 12.566370614359172954 * tot[0];
        part[(size_t)gridDim.x + blockIdx.x] = g.omega * tot[1];
        part[(size_t)2 * gridDim.x + blockIdx.x] = ((g.lpp || g.tri) ? 1.0 : 1.0 / 3.0) * tot[2];
    }
}

// x pass, ftTF variant: forward x -> energies -> v_HL(G) = 4 pi n/G^2 + v_ext
// inverse-x, written over the spectrum.  If keep_n, n(G) is also stored in nG_out.
template <typename PR, bool TRI>
__global__ void k_xhl(GridInfo g, FftAxis ax, typename KT<PR>::C *__restrict__ spec,
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

// x pass, divergence variant: D(G) = v_H(G) + v_ext(G) - sum_a i D_a W_a(G)
// from n(G) and the y-transformed W_a; inverse-x result written over W_0.
template <typename PR, bool TRI>
__global__ void k_xdiv(GridInfo g, FftAxis ax, const typename KT<PR>::C *__restrict__ nG,
                       const typename KT<PR>::C *__restrict__ vext, typename KT<PR>::C *__restrict__ w0,
                       const typename KT<PR>::C *__restrict__ w1, const typename KT<PR>::C *__restrict__ w2)
{
    typedef typename KT<PR>::R R;
    typedef typename KT<PR>::C C;
    typedef typename KT<PR>::CC CC;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx;
    CC *A = reinterpret_cast<CC *>(smraw);
    CC *B = A + nx * g.tk;
    CC *D = B + nx * g.tk;
    ColTile t = col_tile(g, true);
    const RecipB<PR, TRI> rb(g);
    const R fpi = fourpi<PR>();
    const R invN = gcst<PR>(g.invN, g.invNf, g.invN2);
    for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
        const int r = i >> t.tsh, c = i & (t.tk - 1);
        if (c >= t.ncol) continue;
        Gk<R> k = rb.gk(g, r, t.couter[c], t.ckz[c]);
        CC out = cmk<CC>(R(0), R(0));
        if (k.g2 > R(0)) {
            CC n = ldc<PR>(nG[t.cbase[c] + r * t.rstride]);
            CC ve = ldc<PR>(vext[t.cbase[c] + r * t.rstride]);
            R kh;
            if constexpr (TRI) kh = fpi * k.ig2;
            else kh = fpi / k.g2;
            out = cmk<CC>(kh * n.x + ve.x, kh * n.y + ve.y);
        }
        D[i] = out;
    }
    const C *ws[3] = {w0, w1, w2};
    for (int a = 0; a < 3; ++a) {
        load_tile<PR>(ws[a], t, nx, A);
        __syncthreads();
        CC *X = fft_lines<CC, false>(A, B, ax, t.ncol, 1, g.tk, true);
        for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
            const int r = i >> t.tsh, c = i & (t.tk - 1);
            if (c >= t.ncol) continue;
            const R d = rb.d(g, a, r, t.couter[c], t.ckz[c]) * invN;
            CC wv = X[i];
            D[i] = cmk<CC>(D[i].x + d * wv.y, D[i].y - d * wv.x);   // -= i d W
        }
        __syncthreads();
    }
    CC *Y = fft_lines<CC, true>(D, A, ax, t.ncol, 1, g.tk, true);
    store_tile<PR>(w0, t, nx, Y);
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
                 const T *dhat, T c, T s, const void *cs, T *phit, cplx<T> *out, cudaStream_t st)
{
    int P = zpairs_light(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 2 * (size_t)P * g.nz * sizeof(cplx<T>);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
#define CALL(PR)                                                                                          \
    if (mode == 0) k_zfwd<PR, 0><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out);     \
    else if (mode == 1) k_zfwd<PR, 1><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out); \
    else k_zfwd<PR, 2><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
}

template <typename T>
int launch_zgga(const GridInfo &g, const FftAxis &az, cplx<T> *g0, cplx<T> *g1, cplx<T> *g2,
                const T *phit, T temp, const FuncParams &fp, const T *tab, int xc, T *vpart,
                double *part, cudaStream_t st)
{
    int P = zpairs_per_block(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 6 * (size_t)P * g.nz * sizeof(cplx<T>);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
#define CALL(PR) k_zgga<PR, false><<<blocks, th, sm, st>>>(g, az, P, g0, g1, g2, phit, temp, fp, tab, xc, vpart, part)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
    return blocks;
}

int launch_zgga_stress(const GridInfo &g, const FftAxis &az, double2 *g0, double2 *g1, double2 *g2,
                       const double *phit, double temp, const FuncParams &fp, const double *tab, int xc,
                       double *vpart, double *part, cudaStream_t st)
{
    int P = zpairs_per_block(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 6 * (size_t)P * g.nz * sizeof(double2);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
#define CALL(PR) k_zgga<PR, true><<<blocks, th, sm, st>>>(g, az, P, g0, g1, g2, phit, temp, fp, tab, xc, vpart, part)
    OFDFT_DISPATCH(double, g, CALL);
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
int launch_xgrad(const GridInfo &g, const FftAxis &ax, cplx<T> *nspec, const cplx<T> *vext,
                 cplx<T> *g0, cplx<T> *g1, cplx<T> *g2, double *part, cudaStream_t st)
{
    int blocks = tiles_of(g, true);
    size_t sm = 3 * (size_t)g.nx * g.tk * sizeof(cplx<T>);
    int th = g.xth > 0 ? g.xth : threads_for(g.nx * g.tk / 2);
#define CALL(PR)                                                                         \
    if (g.tri) k_xgrad<PR, true><<<blocks, th, sm, st>>>(g, ax, nspec, vext, g0, g1, g2, part); \
    else k_xgrad<PR, false><<<blocks, th, sm, st>>>(g, ax, nspec, vext, g0, g1, g2, part)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
    return blocks;
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

template <typename T>
void launch_xdiv(const GridInfo &g, const FftAxis &ax, const cplx<T> *nG, const cplx<T> *vext,
                 cplx<T> *w0, const cplx<T> *w1, const cplx<T> *w2, cudaStream_t st)
{
    int blocks = tiles_of(g, true);
    size_t sm = 3 * (size_t)g.nx * g.tk * sizeof(cplx<T>);
    int th = g.xth > 0 ? g.xth : threads_for(g.nx * g.tk / 2);
#define CALL(PR)                                                                   \
    if (g.tri) k_xdiv<PR, true><<<blocks, th, sm, st>>>(g, ax, nG, vext, w0, w1, w2); \
    else k_xdiv<PR, false><<<blocks, th, sm, st>>>(g, ax, nG, vext, w0, w1, w2)
    OFDFT_DISPATCH(T, g, CALL);
#undef CALL
}

int xpass_blocks(const GridInfo &g) { return tiles_of(g, true); }

size_t field_smem_max(const GridInfo &g, size_t csize)
{
    int P = zpairs_per_block(g);
    size_t z = 6 * (size_t)P * g.nz * csize;
    size_t y = 2 * (size_t)g.ny * g.tk * csize;
    size_t x = 3 * (size_t)g.nx * g.tk * csize;
    size_t m = z > y ? z : y;
    return m > x ? m : x;
}

namespace {
template <typename PR> cudaError_t smem_limits(int b)
{
    cudaError_t e[] = {
        cudaFuncSetAttribute(k_zfwd<PR, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfwd<PR, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfwd<PR, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zgga<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfinal<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfinal<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_ypass<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_ypass<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xgrad<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xhl<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xdiv<PR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xgrad<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xhl<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xdiv<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return x;
    if constexpr (!std::is_same<PR, float>::value)   // the stress variant (FP64 sets only)
        return cudaFuncSetAttribute(k_zgga<PR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
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
                                 const T *, T, T, const void *, T *, cplx<T> *, cudaStream_t); \
    template int launch_zgga<T>(const GridInfo &, const FftAxis &, cplx<T> *, cplx<T> *,           \
                                cplx<T> *, const T *, T, const FuncParams &, const T *, int, T *, \
                                double *, cudaStream_t);                                          \
    template int launch_zfinal<T>(const GridInfo &, const FftAxis &, bool, const cplx<T> *,        \
                                  const T *, const T *, const T *, const T *, T, T, const void *,   \
                                  T, const FuncParams &, const T *, int, T *, double *,            \
                                  cudaStream_t);                                                  \
    template void launch_ypass<T>(const GridInfo &, const FftAxis &, bool, cplx<T> *, int,         \
                                  long long, cudaStream_t);                                       \
    template int launch_xgrad<T>(const GridInfo &, const FftAxis &, cplx<T> *, const cplx<T> *,    \
                                 cplx<T> *, cplx<T> *, cplx<T> *, double *, cudaStream_t);        \
    template int launch_xhl<T>(const GridInfo &, const FftAxis &, cplx<T> *, const cplx<T> *,      \
                               cplx<T> *, int, double *, cudaStream_t);                          \
    template void launch_xdiv<T>(const GridInfo &, const FftAxis &, const cplx<T> *,               \
                                 const cplx<T> *, cplx<T> *, const cplx<T> *, const cplx<T> *,    \
                                 cudaStream_t);                                                   \
    template cudaError_t set_field_smem_limits<T>(size_t);

OFDFT_INST(double)
OFDFT_INST(float)

}  // namespace ofdft
