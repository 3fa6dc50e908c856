// Batched mixed-radix (2, 3, 4, 5, 8) Stockham FFT on lines held in shared
// memory.  All threads of the block take part; each stage reads one buffer
// and writes the other, with a barrier between stages.
//
// Stage with radix R, Ns = product of earlier radices, for butterfly j of
// n/R:  k = j mod Ns, inputs x[j + r n/R] twiddled by w^{r k n/(Ns R)},
// R-point DFT, outputs to ((j div Ns) Ns R + k) + r Ns.  Forward uses
// w = exp(-2 pi i / n), inverse its conjugate (unnormalised).
#pragma once

#include "ffmath.cuh"
#include "ofdft_internal.h"

namespace ofdft {

// Twiddle tables: cplx<T> at FftAxis::tw, double-float pairs at ::twf.
template <typename C> __device__ __forceinline__ const C *axis_tw(const FftAxis &ax)
{
    return reinterpret_cast<const C *>(ax.tw);
}
template <> __device__ __forceinline__ const ff::cf2 *axis_tw<ff::cf2>(const FftAxis &ax)
{
    return reinterpret_cast<const ff::cf2 *>(ax.twf);
}
template <typename C> __device__ __forceinline__ C ld_tw(const C *p) { return __ldg(p); }
template <> __device__ __forceinline__ ff::cf2 ld_tw<ff::cf2>(const ff::cf2 *p)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    ff::cf2 r;
    r.x = ff::f2(v.x, v.y);
    r.y = ff::f2(v.z, v.w);
    return r;
}

template <typename C, bool INV> __device__ __forceinline__ void dft2(C *v)
{
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <typename C, bool INV> __device__ __forceinline__ void dft4(C *v)
{
    C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    C s13 = cadd(v[1], v[3]), d13 = cmuli<C, INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}

template <typename C, bool INV> __device__ __forceinline__ void dft3(C *v)
{
    typedef decltype(C::x) T;
    constexpr T s3(0.86602540378443864676);   // sin(2 pi/3); constexpr: split at compile time
    constexpr T half(0.5);
    C t1 = cadd(v[1], v[2]);
    C t2 = csub(v[0], cscale(t1, half));
    C t3 = cmuli<C, INV>(cscale(csub(v[1], v[2]), s3));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
}

template <typename C, bool INV> __device__ __forceinline__ void dft5(C *v)
{
    typedef decltype(C::x) T;
    constexpr T c1(0.30901699437494742410), c2(-0.80901699437494742410);
    constexpr T s1(0.95105651629515357212), s2(0.58778525229247312917);
    C p14 = cadd(v[1], v[4]), m14 = csub(v[1], v[4]);
    C p23 = cadd(v[2], v[3]), m23 = csub(v[2], v[3]);
    C a1 = cadd(v[0], cadd(cscale(p14, c1), cscale(p23, c2)));
    C a2 = cadd(v[0], cadd(cscale(p14, c2), cscale(p23, c1)));
    C b1 = cmuli<C, INV>(cadd(cscale(m14, s1), cscale(m23, s2)));
    C b2 = cmuli<C, INV>(csub(cscale(m14, s2), cscale(m23, s1)));
    v[0] = cadd(v[0], cadd(p14, p23));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <typename C, bool INV> __device__ __forceinline__ void dft8(C *v)
{
    typedef decltype(C::x) T;
    constexpr T r(0.70710678118654752440);
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    dft4<C, INV>(e);
    dft4<C, INV>(o);
    // o[k] *= W8^k (forward W8 = exp(-i pi/4))
    o[1] = INV ? cmk<C>(r * (o[1].x - o[1].y), r * (o[1].x + o[1].y))
               : cmk<C>(r * (o[1].x + o[1].y), r * (o[1].y - o[1].x));
    o[2] = cmuli<C, INV>(o[2]);
    o[3] = INV ? cmk<C>(-r * (o[3].x + o[3].y), r * (o[3].x - o[3].y))
               : cmk<C>(r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 4] = csub(e[k], o[k]);
    }
}

template <typename C, int R, bool INV> __device__ __forceinline__ void dftR(C *v)
{
    if (R == 2) dft2<C, INV>(v);
    else if (R == 3) dft3<C, INV>(v);
    else if (R == 4) dft4<C, INV>(v);
    else if (R == 5) dft5<C, INV>(v);
    else dft8<C, INV>(v);
}

// One Stockham stage over nl lines.  Element e of line l lives at
// buf[l * lstride + e * estride].  lines_fast selects whether consecutive
// threads walk lines (column tiles) or butterflies (contiguous lines).
// Column tiles have a power-of-two element stride: their threads then walk
// estride line slots (slots >= nl idle) and take line and butterfly from a
// mask and a shift.  Contiguous lines walk the butterflies in slots rounded
// up to a power of two (slots >= n/R idle).  A power-of-two Ns (every stage
// that follows radix-2, 4 or 8 stages only) splits j the same way; other
// Ns divide.
template <typename C, int R, bool INV>
__device__ __forceinline__ void stage(const C *__restrict__ src, C *__restrict__ dst, int n, int Ns,
                                      const C *__restrict__ tw, int nl, int lstride, int estride,
                                      bool lines_fast)
{
    const int nb = n / R;
    const int tws = n / (Ns * R);
    const bool pslot = lines_fast && (estride & (estride - 1)) == 0;
    const int slots = pslot ? estride : nl;
    const int ssh = __ffs(slots) - 1;
    const int bsh = nb > 1 ? 32 - __clz(nb - 1) : 0;   // butterfly slots 2^bsh >= nb
    const bool pns = (Ns & (Ns - 1)) == 0;
    const int nsh = __ffs(Ns) - 1;
    const int total = lines_fast ? nb * slots : (nl << bsh);
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
        int l, j;
        if (pslot) {
            l = it & (slots - 1);
            j = it >> ssh;
            if (l >= nl) continue;
        } else if (lines_fast) {
            l = it % nl;
            j = it / nl;
        } else {
            j = it & ((1 << bsh) - 1);
            l = it >> bsh;
            if (j >= nb) continue;
        }
        const C *s = src + l * lstride;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[(j + r * nb) * estride];
        const int k = pns ? (j & (Ns - 1)) : j % Ns;
        const int q = pns ? (j >> nsh) : j / Ns;
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = ld_tw(tw + r * k * tws);
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dftR<C, R, INV>(v);
        C *d = dst + l * lstride;
        const int base = q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[(base + r * Ns) * estride] = v[r];
    }
}

// One stage over the lines l0 .. l0 + nlw - 1 that the calling warp owns,
// in a line-major tile (element e of line l at buf[l * lstride + e]); the
// warp's lanes walk the butterflies of each line.
template <typename C, int R, bool INV>
__device__ __forceinline__ void stage_w(const C *__restrict__ src, C *__restrict__ dst, int n, int Ns,
                                        const C *__restrict__ tw, int l0, int nlw, int lstride)
{
    const int nb = n / R;
    const int tws = n / (Ns * R);
    const int bsh = nb > 1 ? 32 - __clz(nb - 1) : 0;
    const bool pns = (Ns & (Ns - 1)) == 0;
    const int nsh = __ffs(Ns) - 1;
    const int total = nlw << bsh;
    for (int it = threadIdx.x & 31; it < total; it += 32) {
        const int j = it & ((1 << bsh) - 1);
        if (j >= nb) continue;
        const int l = l0 + (it >> bsh);
        const C *s = src + l * lstride;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = s[j + r * nb];
        const int k = pns ? (j & (Ns - 1)) : j % Ns;
        const int q = pns ? (j >> nsh) : j / Ns;
        if (k != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                C w = ld_tw(tw + r * k * tws);
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dftR<C, R, INV>(v);
        C *d = dst + l * lstride;
        const int base = q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[base + r * Ns] = v[r];
    }
}

// Full transform of the calling warp's lines (stage_w); stages are
// separated by __syncwarp only, so warps run through their lines
// independently.  The caller synchronises the block before the call (tile
// written by other threads) and before other warps read the result.
// Returns the buffer holding the result (the same for every warp).
template <typename C, bool INV>
__device__ C *fft_lines_w(C *a, C *b, const FftAxis &ax, int l0, int nlw, int lstride)
{
    const C *tw = axis_tw<C>(ax);
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.rad[s], Ns = ax.ns[s];
        switch (R) {
        case 2: stage_w<C, 2, INV>(a, b, ax.n, Ns, tw, l0, nlw, lstride); break;
        case 3: stage_w<C, 3, INV>(a, b, ax.n, Ns, tw, l0, nlw, lstride); break;
        case 4: stage_w<C, 4, INV>(a, b, ax.n, Ns, tw, l0, nlw, lstride); break;
        case 5: stage_w<C, 5, INV>(a, b, ax.n, Ns, tw, l0, nlw, lstride); break;
        default: stage_w<C, 8, INV>(a, b, ax.n, Ns, tw, l0, nlw, lstride); break;
        }
        __syncwarp();
        C *t = a;
        a = b;
        b = t;
    }
    return a;
}

// Full transform of nl lines; data starts in a, b is scratch.  Returns the
// buffer holding the result.  Callers must __syncthreads() before the call
// (data written) and may read the result right after it returns.
template <typename C, bool INV>
__device__ C *fft_lines(C *a, C *b, const FftAxis &ax, int nl, int lstride, int estride, bool lines_fast)
{
    const C *tw = axis_tw<C>(ax);
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.rad[s], Ns = ax.ns[s];
        switch (R) {
        case 2: stage<C, 2, INV>(a, b, ax.n, Ns, tw, nl, lstride, estride, lines_fast); break;
        case 3: stage<C, 3, INV>(a, b, ax.n, Ns, tw, nl, lstride, estride, lines_fast); break;
        case 4: stage<C, 4, INV>(a, b, ax.n, Ns, tw, nl, lstride, estride, lines_fast); break;
        case 5: stage<C, 5, INV>(a, b, ax.n, Ns, tw, nl, lstride, estride, lines_fast); break;
        default: stage<C, 8, INV>(a, b, ax.n, Ns, tw, nl, lstride, estride, lines_fast); break;
        }
        __syncthreads();
        C *t = a;
        a = b;
        b = t;
    }
    return a;
}

// Per-thread accumulator of the FP32 kernels: the running sum is a
// double-float pair (hi + lo, two binary32 words) and each binary32 term
// enters by the DWPlusFP sum of ffmath.cuh (relative error <= 2u^2), so a
// thread's partial carries about 48 significant bits while the FP64 units
// stay idle.  Warps and blocks add the pairs in double-float, and each
// block total is rounded to binary64 once (block_sum_f2); the totals of
// the blocks are added in binary64 by the second reduction stage.
struct AccF {
    ff::f2 v;
    __device__ __forceinline__ AccF() : v(0.0f, 0.0f) {}
    __device__ __forceinline__ explicit AccF(float x) : v(x, 0.0f) {}
    __device__ __forceinline__ AccF &operator+=(float x)
    {
        v = ff::add(v, x);
        return *this;
    }
    __device__ __forceinline__ double value() const { return (double)v.hi + (double)v.lo; }
};

// Per-thread accumulator type of the reductions (AccT<T>::type) and the
// type the terms are formed in (AccT<T>::term): FP64 fields accumulate
// binary64 terms in binary64; FP32 fields accumulate binary32 terms in
// AccF.
template <typename T> struct AccT {
    typedef double type;
    typedef double term;
};
template <> struct AccT<float> {
    typedef AccF type;
    typedef float term;
};

// Deterministic block sum of NQ values; thread 0 returns the totals in tot
// (FP64).  Warp and cross-warp sums in the accumulator type; the block totals
// are added in FP64 by the second reduction stage.
template <int NQ, typename A> __device__ __forceinline__ void block_sum(A *v, double *tot)
{
    __shared__ A red[32][NQ];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        A x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        v[q] = x;
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[wid][q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int q = 0; q < NQ; ++q) {
            A s = A(0);
            for (int w = 0; w < nw; ++w) s += red[w][q];
            tot[q] = (double)s;
        }
    }
    __syncthreads();
}

// In-place form for FP64 accumulators.
template <int NQ> __device__ __forceinline__ void block_sum(double *v)
{
    block_sum<NQ, double>(v, v);
}

// Deterministic block sum of double-float per-thread partials: the warp
// stage adds double-float pairs (shuffles of both words, DWPlusDW), warp 0
// adds the warps' pairs in double-float (lane q sums quantity q in warp
// order) and converts each total to binary64 once; thread 0 returns the
// totals in tot.  The FP64 units see one warp instruction per block: on a
// part whose FP64 rate is 1/64 of FP32, binary64 cross-warp sums had cost
// a visible share of the short field kernels.
template <int NQ> __device__ __forceinline__ void block_sum_f2(const ff::f2 *v, double *tot)
{
    static_assert(NQ <= 32, "one lane per quantity");
    __shared__ float2 red[32][NQ];
    __shared__ double btot[NQ];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        ff::f2 x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ff::f2 y;
            y.hi = __shfl_down_sync(0xffffffffu, x.hi, o);
            y.lo = __shfl_down_sync(0xffffffffu, x.lo, o);
            x = ff::add(x, y);
        }
        if (lane == 0) red[wid][q] = make_float2(x.hi, x.lo);
    }
    __syncthreads();
    if (wid == 0 && lane < NQ) {
        const int nw = (blockDim.x + 31) >> 5;
        ff::f2 s(0.0f, 0.0f);
        for (int w = 0; w < nw; ++w) s = ff::add(s, ff::f2(red[w][lane].x, red[w][lane].y));
        btot[lane] = ff::to_double(s);
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) tot[q] = btot[q];
    __syncthreads();
}

// The FP32 kernels' per-thread partials.
template <int NQ> __device__ __forceinline__ void block_sum(AccF *v, double *tot)
{
    ff::f2 d[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) d[q] = v[q].v;
    block_sum_f2<NQ>(d, tot);
}

}  // namespace ofdft
