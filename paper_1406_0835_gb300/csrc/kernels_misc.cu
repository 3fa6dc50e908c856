// Vector kernels of the CG minimiser, deterministic reductions, the local
// pseudopotential structure factor and forces (Eq. (M12)), the Ewald ion-ion
// terms and the MD integrator.  Every reduction writes per-block partial
// sums that a second kernel adds in a fixed order, so results do not depend
// on scheduling.
#include "fft_core.cuh"
#include "kernels.h"

namespace ofdft {

namespace {

constexpr int kVecThreads = 256;

int vec_blocks(long long n)
{
    long long b = (n + kVecThreads - 1) / kVecThreads;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);   // 8 blocks per SM at most
}

// Blocks of the FP64 vector kernels that also reduce: two per SM, so that
// each thread sums many elements before the block reduction (whose cost is
// per thread, not per element).  The FP32 kernels' double-float partials
// are cheap to reduce, and there the occupancy of vec_blocks wins.
template <typename T> int red_blocks(long long n)
{
    if (sizeof(T) != 8) return vec_blocks(n);
    static const int sms = [] {
        int dev = 0, c = 0;
        return (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && c > 0)
                   ? c
                   : 152;
    }();
    long long b = (n + kVecThreads - 1) / kVecThreads;
    const long long cap = 2LL * sms;
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// Block sum of binary64 per-thread partials through the double-float warp
// stage (block_sum_f2): each partial is split into a double-float pair with
// integer operations (split_int, relative error < 2^-46), so the shuffles and
// adds run on the integer and FP32 units instead of the FP64 ones.
template <int NQ> __device__ __forceinline__ void block_sum_split(const double *v, double *tot)
{
    ff::f2 d[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) d[q] = ff::split_int(v[q]);
    block_sum_f2<NQ>(d, tot);
}
template <int NQ> __device__ __forceinline__ void block_sum_split(AccF *v, double *tot) { block_sum<NQ>(v, tot); }

__global__ void k_reduce(const double *__restrict__ part, int nblk, double *__restrict__ out)
{
    double v[1] = {0.0};
    const double *p = part + (size_t)blockIdx.x * nblk;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) v[0] += p[i];
    block_sum<1>(v);
    if (threadIdx.x == 0) out[blockIdx.x] = v[0];
}

// The reductions of one evaluation in one launch: block q sums row q of the
// x-pass partials (q < 3), of the pointwise partials (GGA, 3 <= q < 9) or
// of the final z-pass partials (the rest) into out[q] (ftTF: out[9 + r] for
// final row r), in the same fixed order as k_reduce.
__global__ void k_reduce_eval(const double *__restrict__ pA, int na, const double *__restrict__ pB, int nb,
                              const double *__restrict__ pC, int nc, int gga, double *__restrict__ out)
{
    const int q = blockIdx.x;
    const double *p;
    int n, o;
    if (q < 3) {
        p = pA + (size_t)q * na;
        n = na;
        o = q;
    } else if (gga && q < 9) {
        p = pB + (size_t)(q - 3) * nb;
        n = nb;
        o = q;
    } else {
        const int r = q - (gga ? 9 : 3);
        p = pC + (size_t)r * nc;
        n = nc;
        o = 9 + r;
    }
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[0] += p[i];
    block_sum<1>(v);
    if (threadIdx.x == 0) out[o] = v[0];
}

template <typename T> __global__ void k_fill(long long n, T *x, T val)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = val;
}

template <typename T> __global__ void k_scale(long long n, T *x, double s, const double *sp)
{
    if (sp != nullptr) s = *sp;
    const T st = (T)s;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        x[i] = x[i] * st;
}

template <typename T, typename U> __global__ void k_convert(long long n, const T *x, U *y)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = (U)x[i];
}

template <typename T> __global__ void k_sumsq(long long n, const T *__restrict__ x, double *part)
{
    typedef typename AccT<T>::type A;
    typedef typename AccT<T>::term P;
    A v[1] = {A(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        P a = (P)x[i];
        v[0] += a * a;
    }
    double tot[1];
    block_sum_split<1>(v, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot[0];
}

template <typename T>
__global__ void k_extrap(long long n, const T *__restrict__ x, const T *__restrict__ xp,
                         T *__restrict__ y, double *part)
{
    double v[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T a = T(2) * x[i] - xp[i];
        y[i] = a;
        v[0] += (double)a * (double)a;
    }
    block_sum<1>(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

template <typename T>
__global__ void k_cg_grad(long long n, const T *__restrict__ phi, const T *__restrict__ v,
                          double mu, const double *mup, T *__restrict__ g,
                          const T *__restrict__ gprev, double *part)
{
    if (mup != nullptr) mu = *mup;
    typedef typename AccT<T>::type A;
    typedef typename AccT<T>::term P;
    const T mut = T(mu);
    A acc[2] = {A(0), A(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T gi = T(2) * phi[i] * (v[i] - mut);
        g[i] = gi;
        acc[0] += (P)gi * (P)gi;
        if (gprev != nullptr) acc[1] += (P)gi * (P)gprev[i];
    }
    double tot[2];
    block_sum_split<2>(acc, tot);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot[0];
        part[gridDim.x + blockIdx.x] = tot[1];
    }
}

template <typename T>
__global__ void k_cg_dir(long long n, const T *__restrict__ g, T *__restrict__ d, double beta,
                         const double *betap, const T *__restrict__ phi, double *part)
{
    if (betap != nullptr) beta = *betap;
    typedef typename AccT<T>::type A;
    typedef typename AccT<T>::term P;
    const P ba = P(beta);
    A acc[5] = {A(0), A(0), A(0), A(0), A(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T gi = g[i];
        T di = (beta == 0.0) ? -gi : (T)(-(P)gi + ba * (P)d[i]);
        d[i] = di;
        P p = (P)phi[i];
        acc[0] += p * (P)di;
        acc[1] += (P)di * (P)di;
        acc[2] += (P)di * (P)gi;
        acc[3] += p * p;
        acc[4] += p * (P)gi;
    }
    double tot[5];
    block_sum_split<5>(acc, tot);
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = tot[q];
}

template <typename T>
__global__ void k_cg_dhat(long long n, const T *__restrict__ g, T *__restrict__ d,
                          const T *__restrict__ phi, const T *__restrict__ v, double c1, double c2,
                          int restart, const double *c12r, T *__restrict__ dhat, double *part)
{
    if (c12r != nullptr) {
        c1 = c12r[0];
        c2 = c12r[1];
        restart = c12r[2] != 0.0;
    }
    typedef typename AccT<T>::type A;
    typedef typename AccT<T>::term P;
    const P c1a = P(c1), c2a = P(c2);
    A acc[1] = {A(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        P di = restart ? -(P)g[i] : (P)d[i] - c1a * (P)phi[i];
        d[i] = (T)di;
        T dh = (T)(c2a * di);
        dhat[i] = dh;
        acc[0] += P(2) * (P)phi[i] * (P)v[i] * (P)dh;
    }
    double tot[1];
    block_sum_split<1>(acc, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot[0];
}

// Truncated Newton: part <- block sums of a.b (binary64).
template <typename T>
__global__ void k_dot(long long n, const T *__restrict__ a, const T *__restrict__ b, double *part)
{
    double v[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[0] += (double)a[i] * (double)b[i];
    double tot[1];
    block_sum_split<1>(v, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot[0];
}

// out = alpha x + beta y (out may alias x or y).
template <typename T>
__global__ void k_axpby(long long n, double alpha, const T *x, double beta, const T *y, T *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (T)(alpha * (double)x[i] + beta * (double)y[i]);
}

// One CG update after a line search: when the device CG state says the
// trial was accepted, phi <- phi_trial, v <- v_trial, g_prev <- g first;
// then g = 2 phi (v - mu) as in k_cg_grad, with the partials sum g^2 and
// sum g.g_prev.  Each element is read once (the accepted trial's phi and v
// feed the gradient directly).
template <typename T>
__global__ void k_cg_update(long long n, const int *__restrict__ accepted, T *__restrict__ phi,
                            const T *__restrict__ phit, T *__restrict__ v, const T *__restrict__ vt,
                            const double *mup, T *__restrict__ g, T *__restrict__ gprev, double *part)
{
    typedef typename AccT<T>::type A;
    typedef typename AccT<T>::term P;
    const bool acc_t = *accepted != 0;
    const T mut = T(*mup);
    A acc[2] = {A(0), A(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T p, vv, go;
        if (acc_t) {
            p = phit[i];
            vv = vt[i];
            go = g[i];
            phi[i] = p;
            v[i] = vv;
            gprev[i] = go;
        } else {
            p = phi[i];
            vv = v[i];
            go = gprev[i];
        }
        T gi = T(2) * p * (vv - mut);
        g[i] = gi;
        acc[0] += (P)gi * (P)gi;
        acc[1] += (P)gi * (P)go;
    }
    double tot[2];
    block_sum_split<2>(acc, tot);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot[0];
        part[gridDim.x + blockIdx.x] = tot[1];
    }
}

// ------------------------------------------------ structure factor, forces
__global__ void k_phases(GridInfo g, int nat, const double *__restrict__ R, double2 *px,
                         double2 *py, double2 *pz)
{
    const int per = g.nx + g.ny + g.K;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nat * per; i += gridDim.x * blockDim.x) {
        const int I = i / per, j = i - I * per;
        double G, r;
        double2 *dst;
        int axis, k;
        if (j < g.nx) {
            k = j <= g.nx / 2 ? j : j - g.nx;
            G = (double)k * g.bx;
            axis = 0;
            dst = px + (size_t)I * g.nx + j;
        } else if (j < g.nx + g.ny) {
            int jj = j - g.nx;
            k = jj <= g.ny / 2 ? jj : jj - g.ny;
            G = (double)k * g.by;
            axis = 1;
            dst = py + (size_t)I * g.ny + jj;
        } else {
            k = j - g.nx - g.ny;
            G = (double)k * g.bz;
            axis = 2;
            dst = pz + (size_t)I * g.K + k;
        }
        r = R[3 * I + axis];
        if (g.tri) {
            // G.R = 2 pi k s_axis with the fractional coordinate s = R Ainv
            G = 6.283185307179586477 * (double)k;
            r = R[3 * I] * g.Ainv[axis] + R[3 * I + 1] * g.Ainv[3 + axis] + R[3 * I + 2] * g.Ainv[6 + axis];
        }
        double s, c;
        sincos(G * r, &s, &c);
        *dst = make_double2(c, -s);      // exp(-i G r)
    }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Local pseudopotential form factor per unit charge, 0 at G = 0.
// Gaussian ion: w(G) = -4 pi exp(-G^2 rc^2/4) / (Omega G^2).
// Heine-Abarenkov, Eq. (E4A), q = |G|, divided by the common charge Z:
// w(q) = -4 pi/(Omega q^2 Z) [(Z - A rc) cos(q rc) + (A/q) sin(q rc)] exp(-(q/qc)^6).
__device__ __forceinline__ double lpp_w(const GridInfo &g, double g2)
{
    if (!(g2 > 0.0)) return 0.0;
    if (g.lpp == 0) return -12.566370614359172954 * exp(-0.25 * g2 * g.rc * g.rc) / (g.omega * g2);
    const double q = sqrt(g2), u = q / g.ha_qc, u2 = u * u;
    double s, c;
    sincos(q * g.rc, &s, &c);
    const double B = (g.ha_Z - g.ha_A * g.rc) * c + g.ha_A * s / q;
    return -12.566370614359172954 * B * exp(-u2 * u2 * u2) / (g.omega * g2 * g.ha_Z);
}

// Pressure weight of the Heine-Abarenkov form per unit charge: the LPP
// pressure is sum_G Re[n*(G) wp(G) sum_I Z_I e^{-iG.R_I}] with
// wp = w + (q/3) dw/dq (Omega w depends on the cell only through q), i.e.
// wp = -4 pi f/(3 Omega q^2 Z) [B + q B' - 6 (q/qc)^6 B],
// q B' = -(Z - A rc) q rc sin(q rc) + A (rc cos(q rc) - sin(q rc)/q).
__device__ __forceinline__ double lpp_wp_ha(const GridInfo &g, double g2)
{
    if (!(g2 > 0.0)) return 0.0;
    const double q = sqrt(g2), u = q / g.ha_qc, u2 = u * u, u6 = u2 * u2 * u2;
    double s, c;
    sincos(q * g.rc, &s, &c);
    const double zc = g.ha_Z - g.ha_A * g.rc;
    const double B = zc * c + g.ha_A * s / q;
    const double qdB = -zc * q * g.rc * s + g.ha_A * (g.rc * c - s / q);
    return -4.1887902047863909846 * exp(-u6) * (B + qdB - 6.0 * u6 * B) / (g.omega * g2 * g.ha_Z);
}

// Pressure weight of either form (Gaussian ion: w (1 - G^2 rc^2/2)/3).
__device__ __forceinline__ double lpp_wp(const GridInfo &g, double g2)
{
    if (g.lpp) return lpp_wp_ha(g, g2);
    return lpp_w(g, g2) * (1.0 - 0.5 * g2 * g.rc * g.rc) * (1.0 / 3.0);
}

// Half-spectrum point (ix, iy, kz): G from the reciprocal basis, Nyquist
// flags, Hermitian weight and the partner G' of the full box that the point
// also stands for (-G, except that an integer index on its Nyquist plane
// keeps +n/2).
struct Hk {
    int ix, iy, kz;
    bool nx_, ny_, nz_;
    double gx, gy, gz, g2, wk;
    double gpx, gpy, gpz, g2p;   // G' and |G'|^2 (= G^2 unless the cell is triclinic)
};

__device__ __forceinline__ Hk hk_at(const GridInfo &g, int ix, int iy, int kz)
{
    Hk h;
    h.ix = ix;
    h.iy = iy;
    h.kz = kz;
    int kx = ix <= g.nx / 2 ? ix : ix - g.nx;
    int ky = iy <= g.ny / 2 ? iy : iy - g.ny;
    h.nx_ = 2 * ix == g.nx;
    h.ny_ = 2 * iy == g.ny;
    h.nz_ = 2 * kz == g.nz;
    const int px = h.nx_ ? kx : -kx, py = h.ny_ ? ky : -ky, pz = h.nz_ ? kz : -kz;
    if (g.tri) {   // G = kx b_0 + ky b_1 + kz b_2
        const double *B = g.Bm;
        h.gx = kx * B[0] + ky * B[3] + kz * B[6];
        h.gy = kx * B[1] + ky * B[4] + kz * B[7];
        h.gz = kx * B[2] + ky * B[5] + kz * B[8];
        h.gpx = px * B[0] + py * B[3] + pz * B[6];
        h.gpy = px * B[1] + py * B[4] + pz * B[7];
        h.gpz = px * B[2] + py * B[5] + pz * B[8];
    } else {
        h.gx = (double)kx * g.bx;
        h.gy = (double)ky * g.by;
        h.gz = (double)kz * g.bz;
        h.gpx = (double)px * g.bx;
        h.gpy = (double)py * g.by;
        h.gpz = (double)pz * g.bz;
    }
    h.g2 = h.gx * h.gx + h.gy * h.gy + h.gz * h.gz;
    h.g2p = h.gpx * h.gpx + h.gpy * h.gpy + h.gpz * h.gpz;
    h.wk = (kz == 0 || h.nz_) ? 1.0 : 2.0;
    return h;
}

// Flat half-spectrum index (< 2^31 for every supported grid) to (ix, iy, kz).
__device__ __forceinline__ Hk hk_flat(const GridInfo &g, int q)
{
    const int kz = q % g.K, r = q / g.K;
    return hk_at(g, r / g.ny, r % g.ny, kz);
}

// v(G) = w(G) sum_I Z_I (P_I + P'_I)/2 with P = exp(-i G.R), P' = exp(i G'.R),
// G' = -G except on Nyquist axes where G'_a = +G_a (the Hermitian partner
// folded onto the stored plane).  Off the Nyquist planes P' = P.
// One block per (ix, iy) row; the row factors Z_I e^{-i(Gx X_I + Gy Y_I)} are
// staged in shared memory in chunks of atoms, and thread kz sums over atoms.
// The Heine-Abarenkov form also writes its pressure weights wp(G) times the
// same sum to vext[NH + q].  In a triclinic cell |G'| differs from |G| on
// the Nyquist planes, so the stored value is the Hermitian part of the
// full-box v, (w(G) P + w(G') P')/2, and the pressure weights (of either
// form) go to vext[NH + q] the same way.
__global__ void k_vext(GridInfo g, int nat, const double *__restrict__ Z,
                       const double2 *__restrict__ px, const double2 *__restrict__ py,
                       const double2 *__restrict__ pz, double2 *__restrict__ vext)
{
    constexpr int kChunk = 256;
    __shared__ double2 a[kChunk], b[kChunk];
    const int ix = blockIdx.x / g.ny, iy = blockIdx.x - ix * g.ny;
    const bool rnyq = (2 * ix == g.nx) || (2 * iy == g.ny);
    double2 acc[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    double2 acc2[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    for (int I0 = 0; I0 < nat; I0 += kChunk) {
        const int nI = min(kChunk, nat - I0);
        __syncthreads();
        for (int j = threadIdx.x; j < nI; j += blockDim.x) {
            const int I = I0 + j;
            double2 u = px[(size_t)I * g.nx + ix], v = py[(size_t)I * g.ny + iy];
            double2 p = zmul(u, v);
            a[j] = make_double2(Z[I] * p.x, Z[I] * p.y);
            if (rnyq) {
                if (2 * ix == g.nx) u.y = -u.y;
                if (2 * iy == g.ny) v.y = -v.y;
                double2 pp = zmul(u, v);
                b[j] = make_double2(Z[I] * pp.x, Z[I] * pp.y);
            }
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kz = threadIdx.x + h * blockDim.x;
            if (kz >= g.K) continue;
            const bool znyq = 2 * kz == g.nz;
            const double2 *pzc = pz + (size_t)I0 * g.K + kz;
            for (int j = 0; j < nI; ++j) {
                double2 c = pzc[(size_t)j * g.K];
                double2 t = zmul(a[j], c);
                acc[h].x += t.x;
                acc[h].y += t.y;
                if (rnyq || znyq) {
                    double2 bb = rnyq ? b[j] : a[j];
                    if (znyq) c.y = -c.y;
                    double2 t2 = zmul(bb, c);
                    acc2[h].x += t2.x;
                    acc2[h].y += t2.y;
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int kz = threadIdx.x + h * blockDim.x;
        if (kz >= g.K) continue;
        Hk k = hk_at(g, ix, iy, kz);
        const size_t q = (size_t)blockIdx.x * g.K + kz;
        if (g.tri) {
            const double2 a1 = acc[h], a2 = (rnyq || k.nz_) ? acc2[h] : acc[h];
            const double w1 = lpp_w(g, k.g2), w2 = lpp_w(g, k.g2p);
            vext[q] = make_double2(0.5 * (w1 * a1.x + w2 * a2.x), 0.5 * (w1 * a1.y + w2 * a2.y));
            const double p1 = lpp_wp(g, k.g2), p2 = lpp_wp(g, k.g2p);
            vext[(size_t)g.NH + q] = make_double2(0.5 * (p1 * a1.x + p2 * a2.x), 0.5 * (p1 * a1.y + p2 * a2.y));
            continue;
        }
        const double w = lpp_w(g, k.g2);
        double2 v = acc[h];
        if (rnyq || k.nz_) v = make_double2(0.5 * (v.x + acc2[h].x), 0.5 * (v.y + acc2[h].y));
        vext[q] = make_double2(w * v.x, w * v.y);
        if (g.lpp) {
            const double wp = lpp_wp_ha(g, k.g2);
            vext[(size_t)g.NH + q] = make_double2(wp * v.x, wp * v.y);
        }
    }
}

// dw/dG^2 per unit charge at fixed Omega w (the strain derivative of the
// form factor): Gaussian ion w (-rc^2/4 - 1/G^2); Heine-Abarenkov from its
// dilation weight, wp = w + (2/3) G^2 dw/dG^2.
__device__ __forceinline__ double lpp_dw(const GridInfo &g, double g2)
{
    if (!(g2 > 0.0)) return 0.0;
    const double w = lpp_w(g, g2);
    if (g.lpp == 0) return w * (-0.25 * g.rc * g.rc - 1.0 / g2);
    return 1.5 * (lpp_wp_ha(g, g2) - w) / g2;
}

// Hartree and local-pseudopotential stress sums of one (ix, iy) row (the
// block's), from the row's structure-factor sums s1 = S(G) and s2 (the
// partner's, on Nyquist rows), thread columns kz = threadIdx.x + h
// blockDim.x; writes the block's 12 partial rows.
__device__ __forceinline__ void gstress_row(const GridInfo &g, int ix, int iy, bool rnyq, const double2 s1[2],
                                            const double2 s2[2], const double2 *__restrict__ nG,
                                            double *__restrict__ part)
{
    double sm[12];
    for (int q = 0; q < 12; ++q) sm[q] = 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int kz = threadIdx.x + h * blockDim.x;
        if (kz >= g.K) continue;
        Hk k = hk_at(g, ix, iy, kz);
        if (!(k.g2 > 0.0)) continue;
        const double2 n = nG[(size_t)blockIdx.x * g.K + kz];
        const double inv = 1.0 / k.g2;
        const double hw = 12.566370614359172954 * (n.x * n.x + n.y * n.y) * inv * inv;
        const double wd = lpp_dw(g, k.g2);
        const double lw = wd * (n.x * s1[h].x + n.y * s1[h].y);
        const double f[6] = {k.gx * k.gx, k.gy * k.gy, k.gz * k.gz, k.gx * k.gy, k.gx * k.gz, k.gy * k.gz};
        for (int q = 0; q < 6; ++q) {
            sm[q] += hw * f[q];
            sm[6 + q] += lw * f[q];
        }
        if (kz > 0 && !k.nz_) {
            const double2 sp = rnyq ? s2[h] : s1[h];
            const double invp = 1.0 / k.g2p;   // |G'| = |G| unless the cell is triclinic
            const double hwp = 12.566370614359172954 * (n.x * n.x + n.y * n.y) * invp * invp;
            const double lp = lpp_dw(g, k.g2p) * (n.x * sp.x + n.y * sp.y);
            const double gx = k.gpx, gy = k.gpy, gz = k.gpz;
            const double fp[6] = {gx * gx, gy * gy, gz * gz, gx * gy, gx * gz, gy * gz};
            for (int q = 0; q < 6; ++q) {
                sm[q] += hwp * fp[q];
                sm[6 + q] += lp * fp[q];
            }
        }
    }
    block_sum<12>(sm);
    if (threadIdx.x == 0)
        for (int q = 0; q < 12; ++q) part[(size_t)q * gridDim.x + blockIdx.x] = sm[q];
}

// Hartree and local-pseudopotential parts of the stress tensor
// (Eq. (StressTensor): homogeneous strain at fixed Omega n(G) and fractional
// coordinates), summed over the full FFT box from the half spectrum:
//   H_ab = sum_G 4 pi |n(G)|^2 G_a G_b / G^4,
//   L_ab = sum_G Re[conj(n(G)) w'(G^2) S(G)] G_a G_b,
// w' = dw/dG^2 per unit charge, S(G) = sum_I Z_I e^{-iG.R_I}.  A point with
// 0 < kz < nz/2 also stands for its partner G' = -G (with +n/2 kept on the
// Nyquist axes): n(G') = conj(n(G)) and conj(S(G')) = sum_I Z_I times the
// phase factors conjugated on the Nyquist axes only, as in k_vext.
// One block per (ix, iy) row; partial rows H xx yy zz xy xz yz, then L.
__global__ void k_gstress(GridInfo g, int nat, const double *__restrict__ Z,
                          const double2 *__restrict__ px, const double2 *__restrict__ py,
                          const double2 *__restrict__ pz, const double2 *__restrict__ nG,
                          double *__restrict__ part)
{
    constexpr int kChunk = 256;
    __shared__ double2 a[kChunk], b[kChunk];
    const int ix = blockIdx.x / g.ny, iy = blockIdx.x - ix * g.ny;
    const bool rnyq = (2 * ix == g.nx) || (2 * iy == g.ny);
    double2 acc[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    double2 acc2[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    for (int I0 = 0; I0 < nat; I0 += kChunk) {
        const int nI = min(kChunk, nat - I0);
        __syncthreads();
        for (int j = threadIdx.x; j < nI; j += blockDim.x) {
            const int I = I0 + j;
            double2 u = px[(size_t)I * g.nx + ix], v = py[(size_t)I * g.ny + iy];
            double2 p = zmul(u, v);
            a[j] = make_double2(Z[I] * p.x, Z[I] * p.y);
            if (rnyq) {
                if (2 * ix == g.nx) u.y = -u.y;
                if (2 * iy == g.ny) v.y = -v.y;
                double2 pp = zmul(u, v);
                b[j] = make_double2(Z[I] * pp.x, Z[I] * pp.y);
            }
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kz = threadIdx.x + h * blockDim.x;
            if (kz >= g.K) continue;
            const double2 *pzc = pz + (size_t)I0 * g.K + kz;
            for (int j = 0; j < nI; ++j) {
                const double2 c = pzc[(size_t)j * g.K];
                double2 t = zmul(a[j], c);
                acc[h].x += t.x;
                acc[h].y += t.y;
                if (rnyq) {
                    double2 t2 = zmul(b[j], c);
                    acc2[h].x += t2.x;
                    acc2[h].y += t2.y;
                }
            }
        }
    }
    gstress_row(g, ix, iy, rnyq, acc, acc2, nG, part);
}

// Per-point weight of the local forces: cn(G) = -Omega w_k w(G) conj(n(G));
// in a triclinic cell without w(G), which k_lpp_forces applies at G and G'.
template <typename T>
__global__ void k_lpp_prep(GridInfo g, const cplx<T> *__restrict__ nG, double2 *__restrict__ cn)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < (int)g.NH; q += gridDim.x * blockDim.x) {
        Hk h = hk_flat(g, q);
        const double s = -g.omega * h.wk * (g.tri ? 1.0 : lpp_w(g, h.g2));
        cplx<T> n = nG[q];
        cn[q] = make_double2(s * (double)n.x, -s * (double)n.y);
    }
}

// F_I,a = -Omega sum_half w_k Re(conj(n(G)) dv_I(G)/dR_I,a),
// dv_I/dR_a = Z_I w(G) (-i G_a P + i G'_a P')/2, i.e. with cn from k_lpp_prep
// F_I,a = Z_I sum G_a Im(cn P) off the Nyquist planes.  Block (atom, chunk).
__global__ void k_lpp_forces(GridInfo g, int nat, const double *__restrict__ Z,
                             const double2 *__restrict__ px, const double2 *__restrict__ py,
                             const double2 *__restrict__ pz, const double2 *__restrict__ cn,
                             double *__restrict__ part)
{
    const int I = blockIdx.x, chunk = blockIdx.y, nchunk = gridDim.y;
    const int NH = (int)g.NH;
    const int per = (NH + nchunk - 1) / nchunk;
    const int q0 = chunk * per;
    const int q1 = min(NH, q0 + per);
    const double2 *pxI = px + (size_t)I * g.nx, *pyI = py + (size_t)I * g.ny, *pzI = pz + (size_t)I * g.K;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        Hk h = hk_flat(g, q);
        double2 a = pxI[h.ix], b = pyI[h.iy], c = pzI[h.kz];
        double2 P = zmul(zmul(a, b), c);
        double2 w = cn[q];
        double imP = w.x * P.y + w.y * P.x;        // Im(cn P)
        double wpart = 1.0;                        // the partner's w(G') in a triclinic cell
        if (g.tri) {
            wpart = lpp_w(g, h.g2p);
            imP *= lpp_w(g, h.g2);
        }
        if (!(h.nx_ || h.ny_ || h.nz_)) {
            acc[0] += h.gx * imP;
            acc[1] += h.gy * imP;
            acc[2] += h.gz * imP;
        } else {
            if (h.nx_) a.y = -a.y;
            if (h.ny_) b.y = -b.y;
            if (h.nz_) c.y = -c.y;
            double2 Pp = zmul(zmul(a, b), c);
            double imPp = (w.x * Pp.y + w.y * Pp.x) * wpart;   // Im(cn P'), with w(G') if triclinic
            // i G'_a P' enters with the opposite sign (G' = -G off the Nyquist planes)
            acc[0] += 0.5 * (h.gx * imP - h.gpx * imPp);
            acc[1] += 0.5 * (h.gy * imP - h.gpy * imPp);
            acc[2] += 0.5 * (h.gz * imP - h.gpz * imPp);
        }
    }
    block_sum<3>(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) part[((size_t)I * nchunk + chunk) * 3 + k] = Z[I] * acc[k];
}

// ----------------------------------------- double-float structure factor
// The FP64 contexts' O(N_G N_at) sums (v_ext and the local forces) in
// double-float arithmetic on the FP32 units (the FP64 unit issues 1/64 of
// their rate); the binary64 kernels above remain for binary64 contexts.
// Products use the complex double-float product (cmul, absolute error a few
// u^2 of the operands' size, u = 2^-24), sums the accurate double-float
// addition.

// Double-float copies of the axis phase tables: pxT[ix][I], pyT[iy][I],
// pzT[kz][I] (atoms fastest, for the force kernel's one-thread-per-atom
// loads) and pzd[I][kz] (for v_ext's one-thread-per-kz loads).
__global__ void k_phase_tables_dd(GridInfo g, int nat, const double2 *__restrict__ px,
                                  const double2 *__restrict__ py, const double2 *__restrict__ pz,
                                  ff::cf2 *pxT, ff::cf2 *pyT, ff::cf2 *pzT, ff::cf2 *pzd)
{
    const int per = g.nx + g.ny + g.K;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nat * per; i += gridDim.x * blockDim.x) {
        const int I = i / per, j = i - I * per;
        double2 v;
        ff::cf2 *dst, *dst2 = nullptr;
        if (j < g.nx) {
            v = px[(size_t)I * g.nx + j];
            dst = pxT + (size_t)j * nat + I;
        } else if (j < g.nx + g.ny) {
            const int jj = j - g.nx;
            v = py[(size_t)I * g.ny + jj];
            dst = pyT + (size_t)jj * nat + I;
        } else {
            const int kz = j - g.nx - g.ny;
            v = pz[(size_t)I * g.K + kz];
            dst = pzT + (size_t)kz * nat + I;
            dst2 = pzd + (size_t)I * g.K + kz;
        }
        ff::cf2 d;
        d.x = ff::from_double(v.x);
        d.y = ff::from_double(v.y);
        *dst = d;
        if (dst2) *dst2 = d;
    }
}

__device__ __forceinline__ ff::cf2 cf2_conj_if(ff::cf2 a, bool c)
{
    if (c) a.y = ff::neg(a.y);
    return a;
}

// Structure-factor sums of one (ix, iy) row in double-float, for thread
// columns kz = threadIdx.x + h blockDim.x (h = 0, 1): s1 = sum_I Z_I px py
// pz, and s2 the partner sum with the phases conjugated on the Nyquist axes
// (rows on an x or y Nyquist plane; with ZNYQ also the kz = nz/2 column).
// The row factors Z_I px py come from the double-float tables in chunks of
// atoms staged in shared memory; thread kz multiplies them by pzd[I][kz].
// Called by every thread of the block.
template <bool ZNYQ>
__device__ __forceinline__ void row_sf_dd(const GridInfo &g, int nat, const double *__restrict__ Z,
                                          const ff::cf2 *__restrict__ pxT, const ff::cf2 *__restrict__ pyT,
                                          const ff::cf2 *__restrict__ pzd, int ix, int iy, double2 s1[2],
                                          double2 s2[2])
{
    constexpr int kChunk = 256;
    __shared__ ff::cf2 a[kChunk], b[kChunk];
    const bool xq = 2 * ix == g.nx, yq = 2 * iy == g.ny, rnyq = xq || yq;
    const ff::f2 z0(0.0f, 0.0f);
    ff::cf2 acc[2] = {{z0, z0}, {z0, z0}}, acc2[2] = {{z0, z0}, {z0, z0}};
    for (int I0 = 0; I0 < nat; I0 += kChunk) {
        const int nI = min(kChunk, nat - I0);
        __syncthreads();
        for (int j = threadIdx.x; j < nI; j += blockDim.x) {
            const int I = I0 + j;
            const ff::cf2 u = pxT[(size_t)ix * nat + I], v = pyT[(size_t)iy * nat + I];
            const ff::f2 zi = ff::split_int(Z[I]);
            ff::cf2 p = ff::cmul(u, v);
            a[j] = {ff::mul(p.x, zi), ff::mul(p.y, zi)};
            if (rnyq) {
                p = ff::cmul(cf2_conj_if(u, xq), cf2_conj_if(v, yq));
                b[j] = {ff::mul(p.x, zi), ff::mul(p.y, zi)};
            }
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kz = threadIdx.x + h * blockDim.x;
            if (kz >= g.K) continue;
            const bool znyq = ZNYQ && 2 * kz == g.nz;
            const ff::cf2 *pzc = pzd + (size_t)I0 * g.K + kz;
            for (int j = 0; j < nI; ++j) {
                const ff::cf2 c = pzc[(size_t)j * g.K];
                const ff::cf2 t = ff::cmul(a[j], c);
                acc[h].x = ff::add(acc[h].x, t.x);
                acc[h].y = ff::add(acc[h].y, t.y);
                if (rnyq || znyq) {
                    const ff::cf2 t2 = ff::cmul(rnyq ? b[j] : a[j], cf2_conj_if(c, znyq));
                    acc2[h].x = ff::add(acc2[h].x, t2.x);
                    acc2[h].y = ff::add(acc2[h].y, t2.y);
                }
            }
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        s1[h] = make_double2(ff::to_double(acc[h].x), ff::to_double(acc[h].y));
        s2[h] = make_double2(ff::to_double(acc2[h].x), ff::to_double(acc2[h].y));
    }
}

// v_ext(G) as k_vext (same Nyquist handling and outputs), with the sums
// over atoms in double-float (row_sf_dd).
__global__ void k_vext_dd(GridInfo g, int nat, const double *__restrict__ Z, const ff::cf2 *__restrict__ pxT,
                          const ff::cf2 *__restrict__ pyT, const ff::cf2 *__restrict__ pzd,
                          double2 *__restrict__ vext)
{
    const int ix = blockIdx.x / g.ny, iy = blockIdx.x - ix * g.ny;
    const bool rnyq = (2 * ix == g.nx) || (2 * iy == g.ny);
    double2 sa[2], sb[2];
    row_sf_dd<true>(g, nat, Z, pxT, pyT, pzd, ix, iy, sa, sb);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int kz = threadIdx.x + h * blockDim.x;
        if (kz >= g.K) continue;
        Hk k = hk_at(g, ix, iy, kz);
        const size_t q = (size_t)blockIdx.x * g.K + kz;
        const double2 s1 = sa[h], s2 = sb[h];
        if (g.tri) {
            const double2 a1 = s1, a2 = (rnyq || k.nz_) ? s2 : s1;
            const double w1 = lpp_w(g, k.g2), w2 = lpp_w(g, k.g2p);
            vext[q] = make_double2(0.5 * (w1 * a1.x + w2 * a2.x), 0.5 * (w1 * a1.y + w2 * a2.y));
            const double p1 = lpp_wp(g, k.g2), p2 = lpp_wp(g, k.g2p);
            vext[(size_t)g.NH + q] = make_double2(0.5 * (p1 * a1.x + p2 * a2.x), 0.5 * (p1 * a1.y + p2 * a2.y));
            continue;
        }
        const double w = lpp_w(g, k.g2);
        double2 v = s1;
        if (rnyq || k.nz_) v = make_double2(0.5 * (v.x + s2.x), 0.5 * (v.y + s2.y));
        vext[q] = make_double2(w * v.x, w * v.y);
        if (g.lpp) {
            const double wp = lpp_wp_ha(g, k.g2);
            vext[(size_t)g.NH + q] = make_double2(wp * v.x, wp * v.y);
        }
    }
}

// Hartree and LPP stress sums as k_gstress, with the structure factor in
// double-float (row_sf_dd; no partner column at kz = nz/2, as there).
__global__ void k_gstress_dd(GridInfo g, int nat, const double *__restrict__ Z, const ff::cf2 *__restrict__ pxT,
                             const ff::cf2 *__restrict__ pyT, const ff::cf2 *__restrict__ pzd,
                             const double2 *__restrict__ nG, double *__restrict__ part)
{
    const int ix = blockIdx.x / g.ny, iy = blockIdx.x - ix * g.ny;
    const bool rnyq = (2 * ix == g.nx) || (2 * iy == g.ny);
    double2 s1[2], s2[2];
    row_sf_dd<false>(g, nat, Z, pxT, pyT, pzd, ix, iy, s1, s2);
    gstress_row(g, ix, iy, rnyq, s1, s2, nG, part);
}

// cn(G) = -Omega w_k w(G) conj(n(G)) as a double-float pair (w included in
// every cell, the partner's w(G') of a triclinic cell is applied by the
// force kernel).
template <typename T>
__global__ void k_lpp_prep_dd(GridInfo g, const cplx<T> *__restrict__ nG, ff::cf2 *__restrict__ cn)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < (int)g.NH; q += gridDim.x * blockDim.x) {
        Hk h = hk_flat(g, q);
        const double s = -g.omega * h.wk * lpp_w(g, h.g2);
        const cplx<T> n = nG[q];
        cn[q] = {ff::from_double(s * (double)n.x), ff::from_double(-s * (double)n.y)};
    }
}

// Local-pseudopotential forces in double-float (same sums as k_lpp_forces):
// F_I,a = Z_I sum_G G_a Im(cn(G) P_I(G)), P_I = px py pz, off the Nyquist
// planes; on them the half-and-half form with the partner G' (conjugated
// phases on the Nyquist axes, w(G') in a triclinic cell).  With G = kx b_0 +
// ky b_1 + kz b_2 the sum is carried as T_j = sum k_j (...) per lattice
// direction and F_I = Z_I sum_j T_j b_j at the end, so the per-point work
// has no G vector.  Block (row chunk, atom chunk), one thread per atom: the
// block walks its rows (ix, iy), stages the row's cn (and the partner
// weights) in shared memory, and each thread runs over kz with its atom's
// row factor px py.  part[(I * gridDim.x + row chunk) * 3 + a].
template <typename T>
__global__ void k_lpp_forces_dd(GridInfo g, int nat, int rows_per_block, const double *__restrict__ Z,
                                const ff::cf2 *__restrict__ pxT, const ff::cf2 *__restrict__ pyT,
                                const ff::cf2 *__restrict__ pzT, const ff::cf2 *__restrict__ cn,
                                const cplx<T> *__restrict__ nG, double *__restrict__ part)
{
    extern __shared__ ff::cf2 scn[];   // [K] row weights, then [K] partner weights (triclinic)
    ff::cf2 *scnp = scn + g.K;
    const int I = blockIdx.y * blockDim.x + threadIdx.x;
    const bool act = I < nat;
    const int nrows = g.nx * g.ny;
    const int r0 = blockIdx.x * rows_per_block, r1 = min(nrows, r0 + rows_per_block);
    const ff::f2 z0(0.0f, 0.0f);
    ff::f2 Tx = z0, Ty = z0, Tz = z0;
    for (int r = r0; r < r1; ++r) {
        const int ix = r / g.ny, iy = r - ix * g.ny;
        const bool xq = 2 * ix == g.nx, yq = 2 * iy == g.ny, rnyq = xq || yq;
        __syncthreads();
        for (int kz = threadIdx.x; kz < g.K; kz += blockDim.x) {
            const size_t q = (size_t)r * g.K + kz;
            scn[kz] = cn[q];
            if (g.tri && (rnyq || 2 * kz == g.nz)) {
                const Hk h = hk_at(g, ix, iy, kz);
                const double s = -g.omega * h.wk * lpp_w(g, h.g2p);
                const cplx<T> n = nG[q];
                scnp[kz] = {ff::from_double(s * (double)n.x), ff::from_double(-s * (double)n.y)};
            }
        }
        __syncthreads();
        if (!act) continue;
        const ff::cf2 u = pxT[(size_t)ix * nat + I], v = pyT[(size_t)iy * nat + I];
        const ff::cf2 ab = ff::cmul(u, v);
        const ff::cf2 abp = rnyq ? ff::cmul(cf2_conj_if(u, xq), cf2_conj_if(v, yq)) : ab;
        ff::f2 A0 = z0, NX = z0, NY = z0, Az = z0;
        const ff::cf2 *pzI = pzT + I;
        for (int kz = 0; kz < g.K; ++kz) {
            const ff::cf2 c = pzI[(size_t)kz * nat];
            const ff::cf2 w = scn[kz];
            const ff::cf2 P = ff::cmul(ab, c);
            const ff::f2 e1 = ff::dot2_sub(w.x, P.y, ff::neg(w.y), P.x);   // Im(w P)
            const bool znyq = 2 * kz == g.nz;
            if (!(rnyq || znyq)) {
                A0 = ff::add(A0, e1);
                Az = ff::add(Az, ff::mul(e1, (float)kz));
            } else {
                const ff::cf2 Pp = ff::cmul(abp, cf2_conj_if(c, znyq));
                const ff::cf2 wp = g.tri ? scnp[kz] : w;
                const ff::f2 e2 = ff::dot2_sub(wp.x, Pp.y, ff::neg(wp.y), Pp.x);   // Im(w' P')
                // (k_j e1 - k'_j e2)/2 with k'_j = k_j on the Nyquist axes, -k_j off them
                const ff::f2 dm = ff::scale(ff::sub(e1, e2), 0.5f), dp = ff::scale(ff::add(e1, e2), 0.5f);
                NX = ff::add(NX, xq ? dm : dp);
                NY = ff::add(NY, yq ? dm : dp);
                Az = ff::add(Az, ff::mul(znyq ? dm : dp, (float)kz));
            }
        }
        const int kx = ix <= g.nx / 2 ? ix : ix - g.nx, ky = iy <= g.ny / 2 ? iy : iy - g.ny;
        Tx = ff::add(Tx, ff::mul(ff::add(A0, NX), (float)kx));
        Ty = ff::add(Ty, ff::mul(ff::add(A0, NY), (float)ky));
        Tz = ff::add(Tz, Az);
    }
    if (!act) return;
    const double t[3] = {ff::to_double(Tx), ff::to_double(Ty), ff::to_double(Tz)};
    double F[3];
    if (g.tri) {
        for (int a = 0; a < 3; ++a) F[a] = t[0] * g.Bm[a] + t[1] * g.Bm[3 + a] + t[2] * g.Bm[6 + a];
    } else {
        F[0] = t[0] * g.bx;
        F[1] = t[1] * g.by;
        F[2] = t[2] * g.bz;
    }
    for (int a = 0; a < 3; ++a) part[((size_t)I * gridDim.x + blockIdx.x) * 3 + a] = Z[I] * F[a];
}

// Sum of force partials: one warp per (atom, component), lanes over the
// chunks in a fixed pattern, then a fixed shuffle tree.
__global__ void k_force_reduce_w(int nat, int nchunk, const double *__restrict__ part, double *F, int accumulate)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= 3 * nat) return;
    const int I = w / 3, k = w - 3 * I;
    double s = 0.0;
    for (int c = lane; c < nchunk; c += 32) s += part[((size_t)I * nchunk + c) * 3 + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) F[w] = accumulate ? F[w] + s : s;
}

// ---------------------------------------------------------------- Ewald
// Separation R_I - R_J reduced to the cell (fractional coordinates in
// [-1/2, 1/2]) and shifted by the lattice vector (a, b, c).
__device__ __forceinline__ void ew_sep(const EwCell &cl, double dx, double dy, double dz, int a, int b, int c,
                                       double &ox, double &oy, double &oz)
{
    if (!cl.tri) {
        const double Lx = cl.a[0], Ly = cl.a[4], Lz = cl.a[8];
        dx -= Lx * rint(dx / Lx);
        dy -= Ly * rint(dy / Ly);
        dz -= Lz * rint(dz / Lz);
        ox = dx - a * Lx;
        oy = dy - b * Ly;
        oz = dz - c * Lz;
        return;
    }
    const double *A = cl.a, *Ai = cl.ai;
    double s0 = dx * Ai[0] + dy * Ai[3] + dz * Ai[6];
    double s1 = dx * Ai[1] + dy * Ai[4] + dz * Ai[7];
    double s2 = dx * Ai[2] + dy * Ai[5] + dz * Ai[8];
    s0 -= rint(s0) + a;
    s1 -= rint(s1) + b;
    s2 -= rint(s2) + c;
    ox = s0 * A[0] + s1 * A[3] + s2 * A[6];
    oy = s0 * A[1] + s1 * A[4] + s2 * A[7];
    oz = s0 * A[2] + s1 * A[5] + s2 * A[8];
}

__global__ void k_ewald_real(int nat, const double *__restrict__ R, const double *__restrict__ Z,
                             EwCell cl, double alpha, double rcut, int3 nimg, double *eion, double *F)
{
    const int I = blockIdx.x;
    const int ix = 2 * nimg.x + 1, iy = 2 * nimg.y + 1, iz = 2 * nimg.z + 1;
    const long long total = (long long)nat * ix * iy * iz;
    const double twosqpi = 1.1283791670955125739;   // 2/sqrt(pi)
    double acc[4] = {0, 0, 0, 0};
    const double xi = R[3 * I], yi = R[3 * I + 1], zi = R[3 * I + 2], ZI = Z[I];
    for (long long q = threadIdx.x; q < total; q += blockDim.x) {
        long long r0 = q;
        const int J = (int)(r0 % nat);
        r0 /= nat;
        const int a = (int)(r0 % ix) - nimg.x;
        r0 /= ix;
        const int b = (int)(r0 % iy) - nimg.y;
        const int c = (int)(r0 / iy) - nimg.z;
        // minimum image of R_I - R_J, then the lattice shift
        double dx, dy, dz;
        ew_sep(cl, xi - R[3 * J], yi - R[3 * J + 1], zi - R[3 * J + 2], a, b, c, dx, dy, dz);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < 1e-24 || r2 >= rcut * rcut) continue;
        double r = sqrt(r2);
        double zz = ZI * Z[J];
        double ec = erfc(alpha * r) / r;
        acc[0] += 0.5 * zz * ec;
        double fm = zz * (ec / r + twosqpi * alpha * exp(-alpha * alpha * r2) / r) / r;
        acc[1] += fm * dx;
        acc[2] += fm * dy;
        acc[3] += fm * dz;
    }
    block_sum<4>(acc);
    if (threadIdx.x == 0) {
        eion[I] = acc[0];
        F[3 * I] = acc[1];
        F[3 * I + 1] = acc[2];
        F[3 * I + 2] = acc[3];
    }
}

// Real-space Ewald stress: per ion I, sum over J and images of
// g(r) r_a r_b / r^2 with g = Z_I Z_J (erfc(a r)/r + (2a/sqrt pi) e^{-a^2 r^2})
// (the pair sum of Sigma_real = -(1/2 Omega) sum' g r_a r_b / r^2), rows
// xx yy zz xy xz yz, one column per ion.  Same pair loop as k_ewald_real.
__global__ void k_ewald_stress_real(int nat, const double *__restrict__ R, const double *__restrict__ Z,
                                    EwCell cl, double alpha, double rcut, int3 nimg, double *part)
{
    const int I = blockIdx.x;
    const int ix = 2 * nimg.x + 1, iy = 2 * nimg.y + 1, iz = 2 * nimg.z + 1;
    const long long total = (long long)nat * ix * iy * iz;
    const double twosqpi = 1.1283791670955125739;   // 2/sqrt(pi)
    double acc[6] = {0, 0, 0, 0, 0, 0};
    const double xi = R[3 * I], yi = R[3 * I + 1], zi = R[3 * I + 2], ZI = Z[I];
    for (long long q = threadIdx.x; q < total; q += blockDim.x) {
        long long r0 = q;
        const int J = (int)(r0 % nat);
        r0 /= nat;
        const int a = (int)(r0 % ix) - nimg.x;
        r0 /= ix;
        const int b = (int)(r0 % iy) - nimg.y;
        const int c = (int)(r0 / iy) - nimg.z;
        double dx, dy, dz;
        ew_sep(cl, xi - R[3 * J], yi - R[3 * J + 1], zi - R[3 * J + 2], a, b, c, dx, dy, dz);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < 1e-24 || r2 >= rcut * rcut) continue;
        double r = sqrt(r2);
        double gr = ZI * Z[J] * (erfc(alpha * r) / r + twosqpi * alpha * exp(-alpha * alpha * r2)) / r2;
        acc[0] += gr * dx * dx;
        acc[1] += gr * dy * dy;
        acc[2] += gr * dz * dz;
        acc[3] += gr * dx * dy;
        acc[4] += gr * dx * dz;
        acc[5] += gr * dy * dz;
    }
    block_sum<6>(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < 6; ++k) part[(size_t)k * nat + I] = acc[k];
}

// Reciprocal Ewald stress from S(G) (k_ewald_S): rows sum wG |S|^2 (the
// reciprocal energy) and sum wG |S|^2 (1/(4 a^2) + 1/G^2) G_a G_b for
// xx yy zz xy xz yz.
__global__ void k_ewald_stress_recip(int nG, const double *__restrict__ Gv, const double *__restrict__ wG,
                                     const double2 *__restrict__ S, double alpha, double *part)
{
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const double q4 = 0.25 / (alpha * alpha);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nG; q += gridDim.x * blockDim.x) {
        const double gx = Gv[3 * q], gy = Gv[3 * q + 1], gz = Gv[3 * q + 2];
        const double2 Sq = S[q];
        const double e = wG[q] * (Sq.x * Sq.x + Sq.y * Sq.y);
        const double c = e * (q4 + 1.0 / (gx * gx + gy * gy + gz * gz));
        acc[0] += e;
        acc[1] += c * gx * gx;
        acc[2] += c * gy * gy;
        acc[3] += c * gz * gz;
        acc[4] += c * gx * gy;
        acc[5] += c * gx * gz;
        acc[6] += c * gy * gz;
    }
    block_sum<7>(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) part[(size_t)k * gridDim.x + blockIdx.x] = acc[k];
}

// S(G) = sum_I Z_I exp(i G.R_I); energy partial sum wG |S|^2.
__global__ void k_ewald_S(int nat, const double *__restrict__ R, const double *__restrict__ Z,
                          int nG, const double *__restrict__ Gv, const double *__restrict__ wG,
                          double2 *S, double *epart)
{
    double acc[1] = {0.0};
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nG; q += gridDim.x * blockDim.x) {
        const double gx = Gv[3 * q], gy = Gv[3 * q + 1], gz = Gv[3 * q + 2];
        double sr = 0.0, si = 0.0;
        for (int I = 0; I < nat; ++I) {
            double s, c;
            sincos(gx * R[3 * I] + gy * R[3 * I + 1] + gz * R[3 * I + 2], &s, &c);
            sr += Z[I] * c;
            si += Z[I] * s;
        }
        S[q] = make_double2(sr, si);
        acc[0] += wG[q] * (sr * sr + si * si);
    }
    block_sum<1>(acc);
    if (threadIdx.x == 0) epart[blockIdx.x] = acc[0];
}

// F_I += 2 Z_I sum_G wG G Im(conj(S(G)) exp(i G.R_I)).
__global__ void k_ewald_F(int nat, const double *__restrict__ R, const double *__restrict__ Z,
                          int nG, const double *__restrict__ Gv, const double *__restrict__ wG,
                          const double2 *__restrict__ S, double *F)
{
    const int I = blockIdx.x;
    double acc[3] = {0, 0, 0};
    for (int q = threadIdx.x; q < nG; q += blockDim.x) {
        const double gx = Gv[3 * q], gy = Gv[3 * q + 1], gz = Gv[3 * q + 2];
        double s, c;
        sincos(gx * R[3 * I] + gy * R[3 * I + 1] + gz * R[3 * I + 2], &s, &c);
        double2 Sq = S[q];
        double im = Sq.x * s - Sq.y * c;        // Im(conj(S) e^{i G.R})
        double f = 2.0 * Z[I] * wG[q] * im;
        acc[0] += f * gx;
        acc[1] += f * gy;
        acc[2] += f * gz;
    }
    block_sum<3>(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) F[3 * I + k] += acc[k];
}

// ------------------------------------------------------------------- MD
// nh[0] = xi (thermostat velocity), nh[1] = eta (its position), nh[2] = K.
__device__ void md_thermo_half(int nat, const double *m, double *V, double h, double kT, double Q,
                               int ndof, double *nh)
{
    double k[1] = {0.0};
    for (int i = threadIdx.x; i < nat; i += blockDim.x)
        k[0] += 0.5 * m[i] * (V[3 * i] * V[3 * i] + V[3 * i + 1] * V[3 * i + 1] + V[3 * i + 2] * V[3 * i + 2]);
    block_sum<1>(k);
    __shared__ double sh[2];
    if (threadIdx.x == 0) {
        double K = k[0];
        double xi = nh[0] + 0.5 * h * (2.0 * K - ndof * kT) / Q;
        double sc = exp(-xi * h);
        nh[1] += xi * h;
        K *= sc * sc;
        xi += 0.5 * h * (2.0 * K - ndof * kT) / Q;
        nh[0] = xi;
        sh[0] = sc;
    }
    __syncthreads();
    const double sc = sh[0];
    for (int i = threadIdx.x; i < 3 * nat; i += blockDim.x) V[i] *= sc;
    __syncthreads();
}

__global__ void k_md_a(int nat, const double *m, double *R, double *V, const double *F, double dt,
                       double kT, double Q, int ndof, int thermo, double *nh)
{
    if (thermo) md_thermo_half(nat, m, V, 0.5 * dt, kT, Q, ndof, nh);
    for (int i = threadIdx.x; i < 3 * nat; i += blockDim.x) {
        V[i] += 0.5 * dt * F[i] / m[i / 3];
        R[i] += dt * V[i];
    }
}

__global__ void k_md_b(int nat, const double *m, double *V, const double *F, double dt, double kT,
                       double Q, int ndof, int thermo, double *nh)
{
    for (int i = threadIdx.x; i < 3 * nat; i += blockDim.x) V[i] += 0.5 * dt * F[i] / m[i / 3];
    __syncthreads();
    if (thermo) md_thermo_half(nat, m, V, 0.5 * dt, kT, Q, ndof, nh);
    double k[1] = {0.0};
    for (int i = threadIdx.x; i < nat; i += blockDim.x)
        k[0] += 0.5 * m[i] * (V[3 * i] * V[3 * i] + V[3 * i + 1] * V[3 * i + 1] + V[3 * i + 2] * V[3 * i + 2]);
    block_sum<1>(k);
    if (threadIdx.x == 0) nh[2] = k[0];
}

// Andersen collisions: ion i with u[i] < prob takes v = sqrt(kT/m_i) xi[i];
// then the kinetic energy into nh[2].  One block.
__global__ void k_andersen(int nat, const double *m, double *V, double kT, double prob,
                           const double *__restrict__ u, const double *__restrict__ xi, double *nh)
{
    for (int i = threadIdx.x; i < nat; i += blockDim.x) {
        if (u[i] < prob) {
            const double sd = sqrt(kT / m[i]);
            for (int a = 0; a < 3; ++a) V[3 * i + a] = sd * xi[3 * i + a];
        }
    }
    __syncthreads();
    double k[1] = {0.0};
    for (int i = threadIdx.x; i < nat; i += blockDim.x)
        k[0] += 0.5 * m[i] * (V[3 * i] * V[3 * i] + V[3 * i + 1] * V[3 * i + 1] + V[3 * i + 2] * V[3 * i + 2]);
    block_sum<1>(k);
    if (threadIdx.x == 0) nh[2] = k[0];
}

}  // namespace

// ---------------------------------------------------------------- launchers
void launch_andersen(int nat, const double *m, double *V, double kT, double prob, const double *u,
                     const double *xi, double *nh, cudaStream_t st)
{
    k_andersen<<<1, 256, 0, st>>>(nat, m, V, kT, prob, u, xi, nh);
}

void launch_reduce(const double *part, int nblk, int nq, double *out, cudaStream_t st)
{
    k_reduce<<<nq, 256, 0, st>>>(part, nblk, out);
}

void launch_reduce_eval(const double *pA, int na, const double *pB, int nb, const double *pC, int nc, bool gga,
                        double *out, cudaStream_t st)
{
    k_reduce_eval<<<gga ? 18 : 12, 256, 0, st>>>(pA, na, pB, nb, pC, nc, gga ? 1 : 0, out);
}

template <typename T> void launch_fill(long long n, T *x, T val, cudaStream_t st)
{
    k_fill<T><<<vec_blocks(n), kVecThreads, 0, st>>>(n, x, val);
}
template <typename T> void launch_scale(long long n, T *x, double s, const double *sp, cudaStream_t st)
{
    k_scale<T><<<vec_blocks(n), kVecThreads, 0, st>>>(n, x, s, sp);
}

template <typename T>
int launch_cg_update(long long n, const int *accepted, T *phi, const T *phit, T *v, const T *vt,
                     const double *mup, T *g, T *gprev, double *part, cudaStream_t st)
{
    int b = red_blocks<T>(n);
    k_cg_update<T><<<b, kVecThreads, 0, st>>>(n, accepted, phi, phit, v, vt, mup, g, gprev, part);
    return b;
}
template <typename T, typename U> void launch_convert(long long n, const T *x, U *y, cudaStream_t st)
{
    k_convert<T, U><<<vec_blocks(n), kVecThreads, 0, st>>>(n, x, y);
}
template <typename T> int launch_sumsq(long long n, const T *x, double *part, cudaStream_t st)
{
    int b = red_blocks<T>(n);
    k_sumsq<T><<<b, kVecThreads, 0, st>>>(n, x, part);
    return b;
}
template <typename T>
int launch_extrap(long long n, const T *x, const T *xp, T *y, double *part, cudaStream_t st)
{
    int b = vec_blocks(n);
    k_extrap<T><<<b, kVecThreads, 0, st>>>(n, x, xp, y, part);
    return b;
}
template <typename T> int launch_dot(long long n, const T *a, const T *b, double *part, cudaStream_t st)
{
    int nb = red_blocks<T>(n);
    k_dot<T><<<nb, kVecThreads, 0, st>>>(n, a, b, part);
    return nb;
}
template <typename T>
void launch_axpby(long long n, double alpha, const T *x, double beta, const T *y, T *out, cudaStream_t st)
{
    k_axpby<T><<<vec_blocks(n), kVecThreads, 0, st>>>(n, alpha, x, beta, y, out);
}

template <typename T>
int launch_cg_grad(long long n, const T *phi, const T *v, double mu, const double *mup, T *g,
                   const T *gprev, double *part, cudaStream_t st)
{
    int b = red_blocks<T>(n);
    k_cg_grad<T><<<b, kVecThreads, 0, st>>>(n, phi, v, mu, mup, g, gprev, part);
    return b;
}
template <typename T>
int launch_cg_dir(long long n, const T *g, T *d, double beta, const double *betap, const T *phi,
                  double *part, cudaStream_t st)
{
    int b = red_blocks<T>(n);
    k_cg_dir<T><<<b, kVecThreads, 0, st>>>(n, g, d, beta, betap, phi, part);
    return b;
}
template <typename T>
int launch_cg_dhat(long long n, const T *g, T *d, const T *phi, const T *v, double c1, double c2,
                   int restart, const double *c12r, T *dhat, double *part, cudaStream_t st)
{
    int b = red_blocks<T>(n);
    k_cg_dhat<T><<<b, kVecThreads, 0, st>>>(n, g, d, phi, v, c1, c2, restart, c12r, dhat, part);
    return b;
}

void launch_phases(const GridInfo &g, int nat, const double *R, double2 *px, double2 *py,
                   double2 *pz, const PhaseTablesDD *dd, cudaStream_t st)
{
    int total = nat * (g.nx + g.ny + g.K);
    int b = (total + 255) / 256;
    k_phases<<<b, 256, 0, st>>>(g, nat, R, px, py, pz);
    if (dd)
        k_phase_tables_dd<<<b, 256, 0, st>>>(g, nat, px, py, pz, (ff::cf2 *)dd->xT, (ff::cf2 *)dd->yT,
                                             (ff::cf2 *)dd->zT, (ff::cf2 *)dd->zd);
}

void launch_vext(const GridInfo &g, int nat, const double *Z, const double2 *px,
                 const double2 *py, const double2 *pz, const PhaseTablesDD *dd, double2 *vext, cudaStream_t st)
{
    int th = 32 * ((g.K + 31) / 32);
    if (th > 128) th = 32 * ((((g.K + 1) / 2) + 31) / 32);    // two columns per thread
    if (dd && g.dd)
        k_vext_dd<<<g.nx * g.ny, th, 0, st>>>(g, nat, Z, (const ff::cf2 *)dd->xT, (const ff::cf2 *)dd->yT,
                                               (const ff::cf2 *)dd->zd, vext);
    else
        k_vext<<<g.nx * g.ny, th, 0, st>>>(g, nat, Z, px, py, pz, vext);
}

namespace {
// Launch shape of the double-float force kernel: one thread per atom in
// blocks of up to 256, rows of the half spectrum split so that about two
// waves of blocks are resident.
struct ForceShape {
    int tpb, achunks, rows_per_block, rchunks;
};
ForceShape force_shape(long long rows, int nat)
{
    ForceShape f;
    const int n = nat > 0 ? nat : 1;
    f.tpb = n >= 256 ? 256 : 32 * ((n + 31) / 32);
    f.achunks = (n + f.tpb - 1) / f.tpb;
    static const int sms = [] {
        int dev = 0, c = 0;
        return (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && c > 0)
                   ? c
                   : 152;
    }();
    const int resident = std::min(32, 2048 / f.tpb);
    long long rc = (2LL * sms * resident + f.achunks - 1) / f.achunks;
    rc = std::max(1LL, std::min(rc, rows));
    f.rows_per_block = (int)((rows + rc - 1) / rc);
    f.rchunks = (int)((rows + f.rows_per_block - 1) / f.rows_per_block);
    return f;
}
}  // namespace

int lpp_force_chunks_dd(long long rows, int nat) { return force_shape(rows, nat).rchunks; }

int lpp_force_chunks(const GridInfo &g, int nat, bool dd)
{
    if (dd && g.dd) return force_shape((long long)g.nx * g.ny, nat).rchunks;
    int nchunk = 1216 / (nat > 0 ? nat : 1);
    if (nchunk < 1) nchunk = 1;
    long long maxc = (g.NH + 1023) / 1024;
    if (nchunk > maxc) nchunk = (int)maxc;
    return nchunk;
}

template <typename T>
int launch_lpp_forces(const GridInfo &g, int nat, const double *Z, const double2 *px,
                      const double2 *py, const double2 *pz, const PhaseTablesDD *dd, const cplx<T> *nG,
                      double2 *cn, double *part, cudaStream_t st)
{
    long long b = (g.NH + 255) / 256;
    const int pb = (int)(b < 4864 ? b : 4864);
    if (dd && g.dd) {
        k_lpp_prep_dd<T><<<pb, 256, 0, st>>>(g, nG, (ff::cf2 *)cn);
        const ForceShape f = force_shape((long long)g.nx * g.ny, nat);
        dim3 grid(f.rchunks, f.achunks);
        k_lpp_forces_dd<T><<<grid, f.tpb, 2 * g.K * sizeof(ff::cf2), st>>>(
            g, nat, f.rows_per_block, Z, (const ff::cf2 *)dd->xT, (const ff::cf2 *)dd->yT,
            (const ff::cf2 *)dd->zT, (const ff::cf2 *)cn, nG, part);
        return f.rchunks;
    }
    k_lpp_prep<T><<<pb, 256, 0, st>>>(g, nG, cn);
    const int nchunk = lpp_force_chunks(g, nat, false);
    dim3 grid(nat, nchunk);
    k_lpp_forces<<<grid, 256, 0, st>>>(g, nat, Z, px, py, pz, cn, part);
    return nchunk;
}

void launch_force_reduce(int nat, int nchunk, const double *part, double *F, int accumulate,
                         cudaStream_t st)
{
    const long long threads = 32LL * 3 * nat;
    k_force_reduce_w<<<(int)((threads + 255) / 256), 256, 0, st>>>(nat, nchunk, part, F, accumulate);
}

void launch_ewald_real(int nat, const double *R, const double *Z, const EwCell &cl, double alpha,
                       double rcut, int3 nimg, double *eion, double *F, cudaStream_t st)
{
    k_ewald_real<<<nat, 256, 0, st>>>(nat, R, Z, cl, alpha, rcut, nimg, eion, F);
}

int launch_ewald_recip(int nat, const double *R, const double *Z, int nG, const double *Gv,
                       const double *wG, double2 *S, double *epart, double *F, cudaStream_t st)
{
    int b = (nG + 255) / 256;
    if (b < 1) b = 1;
    k_ewald_S<<<b, 256, 0, st>>>(nat, R, Z, nG, Gv, wG, S, epart);
    k_ewald_F<<<nat, 256, 0, st>>>(nat, R, Z, nG, Gv, wG, S, F);
    return b;
}

int launch_gstress(const GridInfo &g, int nat, const double *Z, const double2 *px, const double2 *py,
                   const double2 *pz, const PhaseTablesDD *dd, const double2 *nG, double *part, cudaStream_t st)
{
    int th = 32 * ((g.K + 31) / 32);
    if (th > 128) th = 32 * ((((g.K + 1) / 2) + 31) / 32);    // two columns per thread
    if (dd && g.dd)
        k_gstress_dd<<<g.nx * g.ny, th, 0, st>>>(g, nat, Z, (const ff::cf2 *)dd->xT, (const ff::cf2 *)dd->yT,
                                                  (const ff::cf2 *)dd->zd, nG, part);
    else
        k_gstress<<<g.nx * g.ny, th, 0, st>>>(g, nat, Z, px, py, pz, nG, part);
    return g.nx * g.ny;
}

int launch_ewald_stress(int nat, const double *R, const double *Z, const EwCell &cl, double alpha, double rcut,
                        int3 nimg, int nG, const double *Gv, const double *wG, const double2 *S,
                        double *preal, double *precip, cudaStream_t st)
{
    k_ewald_stress_real<<<nat, 256, 0, st>>>(nat, R, Z, cl, alpha, rcut, nimg, preal);
    int b = (nG + 255) / 256;
    if (b < 1) b = 1;
    k_ewald_stress_recip<<<b, 256, 0, st>>>(nG, Gv, wG, S, alpha, precip);
    return b;
}

void launch_md_a(int nat, const double *m, double *R, double *V, const double *F, double dt,
                 double kT, double Q, int ndof, int thermo, double *nh, cudaStream_t st)
{
    k_md_a<<<1, 256, 0, st>>>(nat, m, R, V, F, dt, kT, Q, ndof, thermo, nh);
}

void launch_md_b(int nat, const double *m, double *V, const double *F, double dt, double kT,
                 double Q, int ndof, int thermo, double *nh, cudaStream_t st)
{
    k_md_b<<<1, 256, 0, st>>>(nat, m, V, F, dt, kT, Q, ndof, thermo, nh);
}

#define OFDFT_MISC_INST(T)                                                                         \
    template void launch_fill<T>(long long, T *, T, cudaStream_t);                                 \
    template void launch_scale<T>(long long, T *, double, const double *, cudaStream_t);           \
    template int launch_cg_update<T>(long long, const int *, T *, const T *, T *, const T *,      \
                                     const double *, T *, T *, double *, cudaStream_t);           \
    template int launch_sumsq<T>(long long, const T *, double *, cudaStream_t);                    \
    template int launch_extrap<T>(long long, const T *, const T *, T *, double *, cudaStream_t);   \
    template int launch_dot<T>(long long, const T *, const T *, double *, cudaStream_t);          \
    template void launch_axpby<T>(long long, double, const T *, double, const T *, T *, cudaStream_t); \
    template int launch_cg_grad<T>(long long, const T *, const T *, double, const double *, T *,   \
                                   const T *, double *, cudaStream_t);                            \
    template int launch_cg_dir<T>(long long, const T *, T *, double, const double *, const T *,    \
                                  double *, cudaStream_t);                                        \
    template int launch_cg_dhat<T>(long long, const T *, T *, const T *, const T *, double,       \
                                   double, int, const double *, T *, double *, cudaStream_t);     \
    template int launch_lpp_forces<T>(const GridInfo &, int, const double *, const double2 *,     \
                                      const double2 *, const double2 *, const PhaseTablesDD *,   \
                                      const cplx<T> *, double2 *, double *, cudaStream_t);

OFDFT_MISC_INST(double)
OFDFT_MISC_INST(float)
template void launch_convert<float, double>(long long, const float *, double *, cudaStream_t);
template void launch_convert<double, float>(long long, const double *, float *, cudaStream_t);

}  // namespace ofdft
