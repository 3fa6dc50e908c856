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
#include "fft_core.cuh"
#include "kernels.h"
#include "pointwise.cuh"

namespace ofdft {

namespace {


// G vector of the half-spectrum point (ix, iy, kz) in the accumulator
// precision A, from the per-axis reciprocal spacings (no divisions).
template <typename A> struct Gk {
    A gx, gy, gz, g2;  // G with +n/2 on Nyquist planes
    A dx, dy, dz;      // first-derivative multipliers (0 on the own-axis Nyquist plane)
    A w;               // Hermitian weight of the half spectrum (1 on kz = 0, nz/2)
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

template <typename T> __device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// ------------------------------------------------------------------ z pass
// Pair p of a block holds real lines 2p (real part) and 2p+1 (imaginary part).

template <typename T, int MODE>
__global__ void k_zfwd(GridInfo g, FftAxis az, int P, const T *__restrict__ in,
                       const T *__restrict__ phi, const T *__restrict__ dhat, T c, T s,
                       const void *__restrict__ cs, T *__restrict__ phit,
                       cplx<T> *__restrict__ out)
{
    if (MODE == 2 && cs != nullptr) {   // rotation angle (two T) from the device CG state
        c = reinterpret_cast<const T *>(cs)[0];
        s = reinterpret_cast<const T *>(cs)[1];
    }
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *A = reinterpret_cast<C *>(smraw);
    C *B = A + P * g.nz;
    const long long npairs = (long long)g.nx * g.ny / 2;
    const long long p0 = (long long)blockIdx.x * P;
    const int nl = (int)min((long long)P, npairs - p0);
    const int nz = g.nz, K = g.K;
    const long long base = 2 * p0 * nz;
    for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x) {
        const int line = i / nz, e = i - line * nz;
        T val;
        if (MODE == 0) {
            val = in[base + i];
        } else if (MODE == 1) {
            T ph = phi[base + i];
            val = ph * ph;
        } else {
            T ph = c * phi[base + i] + s * dhat[base + i];
            phit[base + i] = ph;
            val = ph * ph;
        }
        T *dstp = reinterpret_cast<T *>(&A[(line >> 1) * nz + e]);
        dstp[line & 1] = val;
    }
    __syncthreads();
    C *X = fft_lines<C, false>(A, B, az, nl, nz, 1, false);
    const long long obase = 2 * p0 * K;
    for (int i = threadIdx.x; i < 2 * nl * K; i += blockDim.x) {
        const int line = i / K, k = i - line * K;
        const C *row = X + (line >> 1) * nz;
        C z = row[k], zc = cconj(row[k == 0 ? 0 : nz - k]);
        C r = (line & 1) ? cmk<C>(T(0.5) * (z.y - zc.y), T(-0.5) * (z.x - zc.x))
                         : cmk<C>(T(0.5) * (z.x + zc.x), T(0.5) * (z.y + zc.y));
        out[obase + i] = r;
    }
}

// Build the pair-packed complex line C_k = A_k + i B_k (k <= nz/2) and its
// Hermitian completion C_{nz-k} = conj(A_k) + i conj(B_k); the imaginary
// parts of A_0, A_{nz/2} (and B's) are dropped, as a real inverse does.
template <typename C>
__device__ __forceinline__ void pack_c2r(const C *__restrict__ src, long long obase, int nl, int nz,
                                         int K, C *dst)
{
    typedef decltype(C::x) T;
    for (int i = threadIdx.x; i < nl * K; i += blockDim.x) {
        const int p = i / K, k = i - p * K;
        C a = src[obase + (2 * p) * (long long)K + k];
        C b = src[obase + (2 * p + 1) * (long long)K + k];
        if (k == 0 || 2 * k == nz) {
            a.y = T(0);
            b.y = T(0);
        }
        dst[p * nz + k] = cmk<C>(a.x - b.y, a.y + b.x);
        if (k != 0 && 2 * k != nz) dst[p * nz + nz - k] = cmk<C>(a.x + b.y, b.x - a.y);
    }
}

// Unpack a forward-transformed pair-packed line into two half spectra.
template <typename C>
__device__ __forceinline__ void unpack_r2c(const C *X, long long obase, int nl, int nz, int K,
                                           C *__restrict__ out)
{
    typedef decltype(C::x) T;
    for (int i = threadIdx.x; i < 2 * nl * K; i += blockDim.x) {
        const int line = i / K, k = i - line * K;
        const C *row = X + (line >> 1) * nz;
        C z = row[k], zc = cconj(row[k == 0 ? 0 : nz - k]);
        out[obase + i] = (line & 1) ? cmk<C>(T(0.5) * (z.y - zc.y), T(-0.5) * (z.x - zc.x))
                                    : cmk<C>(T(0.5) * (z.x + zc.x), T(0.5) * (z.y + zc.y));
    }
}

// Fused GGA stage: C2R of grad n (3 fields), pointwise functional + XC,
// R2C of W (3 fields, written over grad n).  Partials: F_s, TS, F_xc,
// sum(n df/dn - f), sum W.grad n, sum n(v_xc - eps_xc).
template <typename T>
__global__ void k_zgga(GridInfo g, FftAxis az, int P, cplx<T> *__restrict__ g0,
                       cplx<T> *__restrict__ g1, cplx<T> *__restrict__ g2,
                       const T *__restrict__ phit, T temp, FuncParams fp,
                       const T *__restrict__ tab, int xc, T *__restrict__ vpart,
                       double *__restrict__ part)
{
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nz = g.nz, K = g.K;
    C *buf[4];
    for (int q = 0; q < 4; ++q) buf[q] = reinterpret_cast<C *>(smraw) + q * P * nz;
    const long long npairs = (long long)g.nx * g.ny / 2;
    const long long p0 = (long long)blockIdx.x * P;
    const int nl = (int)min((long long)P, npairs - p0);
    const long long obase = 2 * p0 * K;
    const long long rbase = 2 * p0 * nz;
    C *spec[3] = {g0, g1, g2};
    C *res[3];
    C *scratch = buf[3];
    for (int a = 0; a < 3; ++a) {
        pack_c2r(spec[a], obase, nl, nz, K, buf[a]);
        __syncthreads();
        res[a] = fft_lines<C, true>(buf[a], scratch, az, nl, nz, 1, false);
        if (res[a] == scratch) scratch = buf[a];
    }
    typedef typename AccT<T>::type A;
    A acc[6] = {0, 0, 0, 0, 0, 0};
    const ff::f2 tcoef = ff::from_double(2.0 / OF_K23 * (double)temp);
    for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x) {
        const int line = i / nz, e = i - line * nz;
        const int p = line >> 1, hi = line & 1;
        T gr[3];
        for (int a = 0; a < 3; ++a)   // each thread owns one component of the packed pair
            gr[a] = reinterpret_cast<const T *>(&res[a][p * nz + e])[hi];
        T ph = phit[rbase + i];
        T n = ph * ph;
        T gg = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
        PwOut<T> o = pw_point<T>(fp, tab, tcoef, temp, n, gg, xc);
        const T eps = o.eps, vxc = o.vxc;
        vpart[rbase + i] = o.dfdn + vxc;
        acc[0] += (A)o.f;
        acc[1] += (A)o.ts;
        acc[2] += (A)(n * eps);
        acc[3] += (A)(n * o.dfdn - o.f);
        acc[4] += (A)(o.wc * gg);
        acc[5] += (A)(n * (vxc - eps));
        for (int a = 0; a < 3; ++a) {
            T *d = reinterpret_cast<T *>(&res[a][p * nz + e]);
            d[hi] = o.wc * gr[a];
        }
    }
    __syncthreads();
    // scratch is the one buffer not holding a field
    for (int a = 0; a < 3; ++a) {
        C *X = fft_lines<C, false>(res[a], scratch, az, nl, nz, 1, false);
        unpack_r2c(X, obase, nl, nz, K, spec[a]);
        __syncthreads();
        if (X == scratch) scratch = res[a];
    }
    double tot[6];
    block_sum<6, A>(acc, tot);
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = tot[q];
}

// Final stage: C2R of D(G); v = D(r) + v_part (GGA) or, for ftTF, the
// pointwise functional is evaluated here and added.  Partials (ftTF only
// for the first six): F_s, TS, F_xc, sum(n df/dn - f), 0, sum n(v_xc - eps),
// then sum phi^2 v, sum phi^2, sum 2 phi v dphi/dtheta.
template <typename T, bool FTTF>
__global__ void k_zfinal(GridInfo g, FftAxis az, int P, const cplx<T> *__restrict__ dspec,
                         const T *__restrict__ vpart, const T *__restrict__ phit,
                         const T *__restrict__ phi, const T *__restrict__ dhat, T c, T s,
                         const void *__restrict__ cs, T temp, FuncParams fp,
                         const T *__restrict__ tab, int xc, T *__restrict__ vout,
                         double *__restrict__ part)
{
    if (cs != nullptr) {
        c = reinterpret_cast<const T *>(cs)[0];
        s = reinterpret_cast<const T *>(cs)[1];
    }
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nz = g.nz, K = g.K;
    C *A = reinterpret_cast<C *>(smraw);
    C *B = A + P * nz;
    const long long npairs = (long long)g.nx * g.ny / 2;
    const long long p0 = (long long)blockIdx.x * P;
    const int nl = (int)min((long long)P, npairs - p0);
    const long long obase = 2 * p0 * K;
    const long long rbase = 2 * p0 * nz;
    pack_c2r(dspec, obase, nl, nz, K, A);
    __syncthreads();
    C *X = fft_lines<C, true>(A, B, az, nl, nz, 1, false);
    typedef typename AccT<T>::type Ac;
    Ac acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const ff::f2 tcoef = ff::from_double(2.0 / OF_K23 * (double)temp);
    for (int i = threadIdx.x; i < 2 * nl * nz; i += blockDim.x) {
        const int line = i / nz, e = i - line * nz;
        C d = X[(line >> 1) * nz + e];
        T dr = (line & 1) ? d.y : d.x;
        T ph = phit[rbase + i];
        T n = ph * ph;
        T v;
        if (FTTF) {
            PwOut<T> o = pw_point<T>(fp, tab, tcoef, temp, n, T(0), xc);
            const T eps = o.eps, vxc = o.vxc;
            v = o.dfdn + vxc + dr;
            acc[0] += (Ac)o.f;
            acc[1] += (Ac)o.ts;
            acc[2] += (Ac)(n * eps);
            acc[3] += (Ac)(n * o.dfdn - o.f);
            acc[5] += (Ac)(n * (vxc - eps));
        } else {
            v = vpart[rbase + i] + dr;
        }
        vout[rbase + i] = v;
        acc[6] += (Ac)(n * v);
        acc[7] += (Ac)n;
        if (dhat != nullptr) {
            T dphi = -s * phi[rbase + i] + c * dhat[rbase + i];
            acc[8] += Ac(2) * (Ac)(ph * v) * (Ac)dphi;
        }
    }
    double tot[9];
    block_sum<9, Ac>(acc, tot);
    if (threadIdx.x == 0)
        for (int q = 0; q < 9; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = tot[q];
}

// ------------------------------------------------------------- y/x passes
// Tile: g.tk consecutive kz columns of one ix-plane (y pass) or one iy-row
// (x pass); rows are the transformed axis.

struct ColTile {
    long long base;   // offset of (row 0, kz0) in the field
    long long rstride;
    int kz0, ncol, outer, tk;
};

__device__ __forceinline__ ColTile col_tile(const GridInfo &g, bool xaxis)
{
    const int tk = g.tk;
    const int ntk = (g.K + tk - 1) / tk;
    ColTile t;
    t.tk = tk;
    t.outer = blockIdx.x / ntk;
    t.kz0 = (blockIdx.x - t.outer * ntk) * tk;
    t.ncol = min(tk, g.K - t.kz0);
    if (xaxis) {
        t.base = (long long)t.outer * g.K + t.kz0;   // outer = iy
        t.rstride = (long long)g.ny * g.K;
    } else {
        t.base = (long long)t.outer * g.ny * g.K + t.kz0;  // outer = ix
        t.rstride = g.K;
    }
    return t;
}

template <typename C>
__device__ __forceinline__ void load_tile(const C *__restrict__ src, const ColTile &t, int nrows, C *dst)
{
    for (int i = threadIdx.x; i < nrows * t.tk; i += blockDim.x) {
        const int r = i / t.tk, c = i - r * t.tk;
        if (c < t.ncol) dst[i] = src[t.base + r * t.rstride + c];
    }
}

template <typename C>
__device__ __forceinline__ void store_tile(C *__restrict__ dst, const ColTile &t, int nrows, const C *src)
{
    for (int i = threadIdx.x; i < nrows * t.tk; i += blockDim.x) {
        const int r = i / t.tk, c = i - r * t.tk;
        if (c < t.ncol) dst[t.base + r * t.rstride + c] = src[i];
    }
}

template <typename T, bool INV>
__global__ void k_ypass(GridInfo g, FftAxis ay, cplx<T> *__restrict__ data, long long fstride)
{
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *A = reinterpret_cast<C *>(smraw);
    C *B = A + g.ny * g.tk;
    ColTile t = col_tile(g, false);
    C *f = data + blockIdx.y * fstride;
    load_tile(f, t, g.ny, A);
    __syncthreads();
    C *X = fft_lines<C, INV>(A, B, ay, t.ncol, 1, g.tk, true);
    store_tile(f, t, g.ny, X);
}

// x pass, gradient variant: forward x -> n(G) (stored), energies, then
// i D_a n(G) inverse-x for a = x, y, z.  Partials: E_H, E_loc, P_loc.
template <typename T>
__global__ void k_xgrad(GridInfo g, FftAxis ax, cplx<T> *__restrict__ nspec,
                        const cplx<T> *__restrict__ vext, cplx<T> *__restrict__ g0,
                        cplx<T> *__restrict__ g1, cplx<T> *__restrict__ g2,
                        double *__restrict__ part)
{
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx;
    C *A = reinterpret_cast<C *>(smraw);
    C *B = A + nx * g.tk;
    C *N = B + nx * g.tk;
    ColTile t = col_tile(g, true);
    load_tile(nspec, t, nx, A);
    __syncthreads();
    C *X = fft_lines<C, false>(A, B, ax, t.ncol, 1, g.tk, true);
    typedef typename AccT<T>::type Ac;
    const Ac bx = gsel<Ac>(g.bx, g.bxf), by = gsel<Ac>(g.by, g.byf), bz = gsel<Ac>(g.bz, g.bzf);
    const Ac hr = gsel<Ac>(g.hr, g.hrf);
    const T invN = gsel<T>(g.invN, g.invNf);
    Ac acc[3] = {0, 0, 0};     // sum w |n|^2/G^2, sum w Re(n* v_ext), sum w Re(n* v_ext)(1 - G^2 rc^2/2)
    for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
        const int r = i / g.tk, c = i - r * g.tk;
        if (c >= t.ncol) continue;
        C nG = cscale(X[i], invN);
        N[i] = nG;
        Gk<Ac> k = gvec<Ac>(g, bx, by, bz, r, t.outer, t.kz0 + c);
        if (k.g2 > Ac(0)) {
            C ve = vext[t.base + r * t.rstride + c];
            Ac n2 = (Ac)nG.x * nG.x + (Ac)nG.y * nG.y;
            Ac re = (Ac)nG.x * ve.x + (Ac)nG.y * ve.y;
            acc[0] += k.w * n2 / k.g2;
            acc[1] += k.w * re;
            acc[2] += k.w * re * (Ac(1) - hr * k.g2);
        }
    }
    __syncthreads();
    store_tile(nspec, t, nx, N);
    C *outs[3] = {g0, g1, g2};
    for (int a = 0; a < 3; ++a) {
        for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
            const int r = i / g.tk, c = i - r * g.tk;
            Gk<Ac> k = gvec<Ac>(g, bx, by, bz, r, t.outer, t.kz0 + min(c, t.ncol - 1));
            T d = T(a == 0 ? k.dx : (a == 1 ? k.dy : k.dz));
            C v = N[i];
            A[i] = cmk<C>(-d * v.y, d * v.x);      // i D_a n(G)
        }
        __syncthreads();
        C *Y = fft_lines<C, true>(A, B, ax, t.ncol, 1, g.tk, true);
        store_tile(outs[a], t, nx, Y);
        __syncthreads();
    }
    double tot[3];
    block_sum<3, Ac>(acc, tot);
    if (threadIdx.x == 0) {
        // E_H = (Omega/2) sum 4 pi |n|^2/G^2, E_loc = Omega sum Re(n* v_ext),
        // P_loc = (1/3) sum Re(n* v_ext)(1 - G^2 rc^2/2)
        part[blockIdx.x] = 0.5 * g.omega * 12.566370614359172954 * tot[0];
        part[(size_t)gridDim.x + blockIdx.x] = g.omega * tot[1];
        part[(size_t)2 * gridDim.x + blockIdx.x] = (1.0 / 3.0) * tot[2];
    }
}

// x pass, ftTF variant: forward x -> energies -> v_HL(G) = 4 pi n/G^2 + v_ext
// inverse-x, written over the spectrum.  If keep_n, n(G) is also stored in nG_out.
template <typename T>
__global__ void k_xhl(GridInfo g, FftAxis ax, cplx<T> *__restrict__ spec,
                      const cplx<T> *__restrict__ vext, cplx<T> *__restrict__ nG_out,
                      int inverse, double *__restrict__ part)
{
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx;
    C *A = reinterpret_cast<C *>(smraw);
    C *B = A + nx * g.tk;
    ColTile t = col_tile(g, true);
    load_tile(spec, t, nx, A);
    __syncthreads();
    C *X = fft_lines<C, false>(A, B, ax, t.ncol, 1, g.tk, true);
    typedef typename AccT<T>::type Ac;
    const Ac bx = gsel<Ac>(g.bx, g.bxf), by = gsel<Ac>(g.by, g.byf), bz = gsel<Ac>(g.bz, g.bzf);
    const Ac hr = gsel<Ac>(g.hr, g.hrf);
    const Ac fourpi = gsel<Ac>(12.566370614359172954, 12.566370614359172954f);
    const T invN = gsel<T>(g.invN, g.invNf);
    Ac acc[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
        const int r = i / g.tk, c = i - r * g.tk;
        if (c >= t.ncol) continue;
        C nG = cscale(X[i], invN);
        Gk<Ac> k = gvec<Ac>(g, bx, by, bz, r, t.outer, t.kz0 + c);
        C ve = vext[t.base + r * t.rstride + c];
        C out = cmk<C>(T(0), T(0));
        if (k.g2 > Ac(0)) {
            Ac n2 = (Ac)nG.x * nG.x + (Ac)nG.y * nG.y;
            Ac re = (Ac)nG.x * ve.x + (Ac)nG.y * ve.y;
            acc[0] += k.w * n2 / k.g2;
            acc[1] += k.w * re;
            acc[2] += k.w * re * (Ac(1) - hr * k.g2);
            T kh = T(fourpi / k.g2);
            out = cmk<C>(kh * nG.x + ve.x, kh * nG.y + ve.y);
        }
        if (nG_out != nullptr) nG_out[t.base + r * t.rstride + c] = nG;
        X[i] = out;
    }
    __syncthreads();
    if (inverse) {
        C *other = (X == A) ? B : A;
        C *Y = fft_lines<C, true>(X, other, ax, t.ncol, 1, g.tk, true);
        store_tile(spec, t, nx, Y);
    }
    double tot[3];
    block_sum<3, Ac>(acc, tot);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = 0.5 * g.omega * 12.566370614359172954 * tot[0];
        part[(size_t)gridDim.x + blockIdx.x] = g.omega * tot[1];
        part[(size_t)2 * gridDim.x + blockIdx.x] = (1.0 / 3.0) * tot[2];
    }
}

// x pass, divergence variant: D(G) = v_H(G) + v_ext(G) - sum_a i D_a W_a(G)
// from n(G) and the y-transformed W_a; inverse-x result written over W_0.
template <typename T>
__global__ void k_xdiv(GridInfo g, FftAxis ax, const cplx<T> *__restrict__ nG,
                       const cplx<T> *__restrict__ vext, cplx<T> *__restrict__ w0,
                       const cplx<T> *__restrict__ w1, const cplx<T> *__restrict__ w2)
{
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nx = g.nx;
    C *A = reinterpret_cast<C *>(smraw);
    C *B = A + nx * g.tk;
    C *D = B + nx * g.tk;
    ColTile t = col_tile(g, true);
    typedef typename AccT<T>::type Ac;
    const Ac bx = gsel<Ac>(g.bx, g.bxf), by = gsel<Ac>(g.by, g.byf), bz = gsel<Ac>(g.bz, g.bzf);
    const Ac fourpi = gsel<Ac>(12.566370614359172954, 12.566370614359172954f);
    const T invN = gsel<T>(g.invN, g.invNf);
    for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
        const int r = i / g.tk, c = i - r * g.tk;
        if (c >= t.ncol) continue;
        Gk<Ac> k = gvec<Ac>(g, bx, by, bz, r, t.outer, t.kz0 + c);
        C out = cmk<C>(T(0), T(0));
        if (k.g2 > Ac(0)) {
            C n = nG[t.base + r * t.rstride + c];
            C ve = vext[t.base + r * t.rstride + c];
            T kh = T(fourpi / k.g2);
            out = cmk<C>(kh * n.x + ve.x, kh * n.y + ve.y);
        }
        D[i] = out;
    }
    const C *ws[3] = {w0, w1, w2};
    for (int a = 0; a < 3; ++a) {
        load_tile(ws[a], t, nx, A);
        __syncthreads();
        C *X = fft_lines<C, false>(A, B, ax, t.ncol, 1, g.tk, true);
        for (int i = threadIdx.x; i < nx * g.tk; i += blockDim.x) {
            const int r = i / g.tk, c = i - r * g.tk;
            if (c >= t.ncol) continue;
            Gk<Ac> k = gvec<Ac>(g, bx, by, bz, r, t.outer, t.kz0 + c);
            T d = T(a == 0 ? k.dx : (a == 1 ? k.dy : k.dz)) * invN;
            C wv = X[i];
            D[i] = cmk<C>(D[i].x + d * wv.y, D[i].y - d * wv.x);   // -= i d W
        }
        __syncthreads();
    }
    C *Y = fft_lines<C, true>(D, A, ax, t.ncol, 1, g.tk, true);
    store_tile(w0, t, nx, Y);
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

int threads_for(int work)
{
    int t = 64;
    while (t < 256 && t < work) t *= 2;
    return t;
}

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_zfwd(const GridInfo &g, const FftAxis &az, int mode, const T *in, const T *phi,
                 const T *dhat, T c, T s, const void *cs, T *phit, cplx<T> *out, cudaStream_t st)
{
    int P = zpairs_per_block(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 2 * (size_t)P * g.nz * sizeof(cplx<T>);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
    if (mode == 0) k_zfwd<T, 0><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out);
    else if (mode == 1) k_zfwd<T, 1><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out);
    else k_zfwd<T, 2><<<blocks, th, sm, st>>>(g, az, P, in, phi, dhat, c, s, cs, phit, out);
}

template <typename T>
int launch_zgga(const GridInfo &g, const FftAxis &az, cplx<T> *g0, cplx<T> *g1, cplx<T> *g2,
                const T *phit, T temp, const FuncParams &fp, const T *tab, int xc, T *vpart,
                double *part, cudaStream_t st)
{
    int P = zpairs_per_block(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 4 * (size_t)P * g.nz * sizeof(cplx<T>);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
    k_zgga<T><<<blocks, th, sm, st>>>(g, az, P, g0, g1, g2, phit, temp, fp, tab, xc, vpart, part);
    return blocks;
}

template <typename T>
int launch_zfinal(const GridInfo &g, const FftAxis &az, bool fttf, const cplx<T> *dspec,
                  const T *vpart, const T *phit, const T *phi, const T *dhat, T c, T s,
                  const void *cs, T temp, const FuncParams &fp, const T *tab, int xc, T *vout,
                  double *part, cudaStream_t st)
{
    int P = zpairs_per_block(g);
    long long npairs = (long long)g.nx * g.ny / 2;
    int blocks = (int)((npairs + P - 1) / P);
    size_t sm = 2 * (size_t)P * g.nz * sizeof(cplx<T>);
    int th = g.zth > 0 ? g.zth : threads_for(P * g.nz);
    if (fttf)
        k_zfinal<T, true><<<blocks, th, sm, st>>>(g, az, P, dspec, vpart, phit, phi, dhat, c, s,
                                                  cs, temp, fp, tab, xc, vout, part);
    else
        k_zfinal<T, false><<<blocks, th, sm, st>>>(g, az, P, dspec, vpart, phit, phi, dhat, c, s,
                                                   cs, temp, fp, tab, xc, vout, part);
    return blocks;
}

template <typename T>
void launch_ypass(const GridInfo &g, const FftAxis &ay, bool inv, cplx<T> *data, int nfields,
                  long long fstride, cudaStream_t st)
{
    int ntk = (g.K + g.tk - 1) / g.tk;
    dim3 grid(g.nx * ntk, nfields);
    size_t sm = 2 * (size_t)g.ny * g.tk * sizeof(cplx<T>);
    int th = g.xth > 0 ? g.xth : threads_for(g.ny * g.tk / 2);
    if (inv) k_ypass<T, true><<<grid, th, sm, st>>>(g, ay, data, fstride);
    else k_ypass<T, false><<<grid, th, sm, st>>>(g, ay, data, fstride);
}

template <typename T>
int launch_xgrad(const GridInfo &g, const FftAxis &ax, cplx<T> *nspec, const cplx<T> *vext,
                 cplx<T> *g0, cplx<T> *g1, cplx<T> *g2, double *part, cudaStream_t st)
{
    int ntk = (g.K + g.tk - 1) / g.tk;
    int blocks = g.ny * ntk;
    size_t sm = 3 * (size_t)g.nx * g.tk * sizeof(cplx<T>);
    int th = g.xth > 0 ? g.xth : threads_for(g.nx * g.tk / 2);
    k_xgrad<T><<<blocks, th, sm, st>>>(g, ax, nspec, vext, g0, g1, g2, part);
    return blocks;
}

template <typename T>
int launch_xhl(const GridInfo &g, const FftAxis &ax, cplx<T> *spec, const cplx<T> *vext,
               cplx<T> *nG_out, int inverse, double *part, cudaStream_t st)
{
    int ntk = (g.K + g.tk - 1) / g.tk;
    int blocks = g.ny * ntk;
    size_t sm = 2 * (size_t)g.nx * g.tk * sizeof(cplx<T>);
    int th = g.xth > 0 ? g.xth : threads_for(g.nx * g.tk / 2);
    k_xhl<T><<<blocks, th, sm, st>>>(g, ax, spec, vext, nG_out, inverse, part);
    return blocks;
}

template <typename T>
void launch_xdiv(const GridInfo &g, const FftAxis &ax, const cplx<T> *nG, const cplx<T> *vext,
                 cplx<T> *w0, const cplx<T> *w1, const cplx<T> *w2, cudaStream_t st)
{
    int ntk = (g.K + g.tk - 1) / g.tk;
    int blocks = g.ny * ntk;
    size_t sm = 3 * (size_t)g.nx * g.tk * sizeof(cplx<T>);
    int th = g.xth > 0 ? g.xth : threads_for(g.nx * g.tk / 2);
    k_xdiv<T><<<blocks, th, sm, st>>>(g, ax, nG, vext, w0, w1, w2);
}

size_t field_smem_max(const GridInfo &g, size_t csize)
{
    int P = zpairs_per_block(g);
    size_t z = 4 * (size_t)P * g.nz * csize;
    size_t y = 2 * (size_t)g.ny * g.tk * csize;
    size_t x = 3 * (size_t)g.nx * g.tk * csize;
    size_t m = z > y ? z : y;
    return m > x ? m : x;
}

template <typename T> cudaError_t set_field_smem_limits(size_t bytes)
{
    int b = (int)bytes;
    cudaError_t e[] = {
        cudaFuncSetAttribute(k_zfwd<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfwd<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfwd<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zgga<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfinal<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_zfinal<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_ypass<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_ypass<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xgrad<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xhl<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
        cudaFuncSetAttribute(k_xdiv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, b)};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
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
