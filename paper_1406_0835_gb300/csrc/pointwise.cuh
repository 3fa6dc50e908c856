// Pointwise finite-T functional math, shared by host (checks) and device.
//
//   tfunc_eval   xi, zeta, A, B of t and their t-derivatives from the table
//   enhance      F(x) and dF/dx of the enhancement factors (Sec. III B)
//   fs_point     f_s, df_s/dn and W = df_s/d(grad n) / grad n at one point
//                (Eqs. (fTF), (vTF), (FGGA), (s_s), (s_0defn), (vftGGA))
//   pz81_point   Perdew-Zunger LDA eps_xc and v_xc (Sec. IV, Eq. (vxc1) at T = 0)
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

#include "ffmath.cuh"
#include "ofdft_internal.h"

namespace ofdft {

#ifdef __CUDACC__
#define OF_HD __host__ __device__ __forceinline__
#else
#define OF_HD inline
#endif

// t = m 2^e with m in [1, 2); returns m and 2^-e.
OF_HD double split_pow2(double t, int &e, double &inv2e)
{
    int64_t b;
#ifdef __CUDA_ARCH__
    b = __double_as_longlong(t);
#else
    memcpy(&b, &t, 8);
#endif
    e = (int)((b >> 52) & 0x7ff) - 1023;
    int64_t mb = (b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL;
    int64_t ib = (int64_t)(1023 - e) << 52;
    double m;
#ifdef __CUDA_ARCH__
    m = __longlong_as_double(mb);
    inv2e = __longlong_as_double(ib);
#else
    memcpy(&m, &mb, 8);
    memcpy(&inv2e, &ib, 8);
#endif
    return m;
}

OF_HD float split_pow2(float t, int &e, float &inv2e)
{
    int32_t b;
#ifdef __CUDA_ARCH__
    b = __float_as_int(t);
#else
    memcpy(&b, &t, 4);
#endif
    e = (int)((b >> 23) & 0xff) - 127;
    int32_t mb = (b & 0x007fffff) | 0x3f800000;
    int32_t ib = (int32_t)(127 - e) << 23;
    float m;
#ifdef __CUDA_ARCH__
    m = __int_as_float(mb);
    inv2e = __int_as_float(ib);
#else
    memcpy(&m, &mb, 4);
    memcpy(&inv2e, &ib, 4);
#endif
    return m;
}

// n^{-1/3} for n > 0: seed from the exponent split n = m 2^(3q + r), m 2^r in
// [1, 8), with a single-precision power of that factor, then Newton steps
// y <- y (4 - n y^3)/3 (quadratic convergence; 2 steps reach double rounding
// from a ~1e-7 seed, 1 step reaches float rounding).
OF_HD double inv_cbrt(double n)
{
    int e;
    double s;
    double m = split_pow2(n, e, s);
    int q = (e >= 0) ? e / 3 : -((2 - e) / 3);      // floor(e / 3)
    int r = e - 3 * q;                                 // 0, 1, 2
    double mm = m * (double)(1 << r);
    double y = (double)powf((float)mm, -1.0f / 3.0f);
    int64_t ib = (int64_t)(1023 - q) << 52;            // 2^-q
    double sc;
#ifdef __CUDA_ARCH__
    sc = __longlong_as_double(ib);
#else
    memcpy(&sc, &ib, 8);
#endif
    y *= sc;
    for (int k = 0; k < 2; ++k) y = y * (4.0 - n * (y * y * y)) * (1.0 / 3.0);
    return y;
}

OF_HD float inv_cbrt(float n)
{
    float y = powf(n, -1.0f / 3.0f);
    return y * (4.0f - n * (y * y * y)) * (1.0f / 3.0f);
}

// out[0..3] = xi, zeta, A, B; out[4..7] = d/dt of each (nf functions: 2 or 4).
template <typename T, int NF = kTfFuncs>
OF_HD void tfunc_eval(const T *__restrict__ tab, T t, T out[8])
{
    const T pi2 = T(9.8696044010893586188);
    if (!(t >= T(9.5367431640625e-07))) {            // t < 2^-20: Sommerfeld limit
        T t2 = t * t;
        out[0] = T(1) + T(5.0 / 12.0) * pi2 * t2;     // xi = 1 + (5 pi^2/12) t^2
        out[1] = T(5.0 / 6.0) * pi2 * t2;             // zeta = (5 pi^2/6) t^2
        out[2] = T(1) - T(0.75) * pi2 * t2;           // A = 1 - (3 pi^2/4) t^2
        out[3] = T(0.8);                              // B -> 4/5
        out[4] = T(5.0 / 6.0) * pi2 * t;
        out[5] = T(5.0 / 3.0) * pi2 * t;
        out[6] = T(-1.5) * pi2 * t;
        out[7] = T(0);
        return;
    }
    if (t >= T(17179869184.0)) {                      // t >= 2^34: classical gas
        // e^eta = (4/(3 sqrt(pi))) t^{-3/2}; xi = (5/2) t; zeta = (5/3) t (5/2 - eta); h~ = 3
        T eta = T(-0.28468287047291918) - T(1.5) * log(t);
        out[0] = T(2.5) * t;
        out[1] = T(5.0 / 3.0) * t * (T(2.5) - eta);
        out[2] = T(1.2) / t;
        out[3] = T(0);
        out[4] = T(2.5);
        out[5] = T(5.0 / 3.0) * (T(2.5) - eta) + T(2.5);
        out[6] = T(-1.2) / (t * t);
        out[7] = T(0);
        return;
    }
    int e;
    T inv2e;
    T m = split_pow2(t, e, inv2e);
    int sub = (int)((m - T(1)) * T(4));
    T u = T(8) * (m - T(1)) - T(2 * sub + 1);
    const T *c = tab + ((size_t)((e - kTfEmin) * kTfSub + sub) * kTfFuncs) * kTfNc;
    T dudt = T(8) * inv2e;
#pragma unroll
    for (int q = 0; q < NF; ++q) {
        const T *cq = c + q * kTfNc;
        T p = cq[kTfDeg], dp = T(0);
#pragma unroll
        for (int j = kTfDeg - 1; j >= 0; --j) {
            dp = dp * u + p;
            p = p * u + cq[j];
        }
        out[q] = p;
        out[4 + q] = dp * dudt;
    }
}

// Enhancement factor F(x), x = s^2, and dF/dx.
template <typename T>
OF_HD void enhance(const FuncParams &fp, T x, T &F, T &dF)
{
    if (fp.kind == 1) {                       // SGA form, Eq. (SGA-F)
        F = T(1) + T(fp.p0) * x;
        dF = T(fp.p0);
    } else if (fp.kind == 3) {                // KST2 form, Eq. (KST2F)
        T den = T(1) / (T(1) + T(fp.p1) * x);
        F = T(1) + T(fp.p0) * x * den;
        dF = T(fp.p0) * den * den;
    } else {                                  // VT84F, Eq. (VT84F), m = 8, n = 4
        const T mu = T(2.778), al = T(1.2965);
        const T tiny = sizeof(T) == 8 ? T(1e-100) : T(1e-15);
        if (x <= tiny) {                      // removable 0/0 at x = 0
            F = T(1);
            dF = -mu + al + T(5.0 / 3.0);
            return;
        }
        T e1 = exp(-al * x);
        T x2 = x * x;
        T em = -expm1(-al * x2);              // 1 - exp(-al x^2)
        T q = T(1) + mu * x;
        T inv = T(1) / (x * q);               // one division for 1/x and 1/(1 + mu x)
        T rx = q * inv;
        T den = x * inv;
        F = T(1) - mu * x * e1 * den + em * (rx - T(1)) + T(5.0 / 3.0) * x;
        dF = -mu * e1 * (T(1) - al * x - al * mu * x2) * den * den
             + T(2) * al * (T(1) - em) * (T(1) - x) - em * rx * rx + T(5.0 / 3.0);
    }
}

// Output of the non-interacting functional at one point.
template <typename T> struct FsOut {
    T f;      // f_s
    T ts;     // tau0 zeta F_sigma (entropic density T s)
    T dfdn;   // partial f / partial n (without the divergence term)
    T wc;     // W = wc * grad n
    T y13;    // n^{-1/3} (reused by the XC term)
};

// Constants: C_TF = (3/10)(3 pi^2)^{2/3}; (3 pi^2)^{2/3}; cs = 1/(4 (3 pi^2)^{2/3}).
#define OF_K23 9.5707800006273045              /* (3 pi^2)^{2/3} */
#define OF_CTF (0.3 * OF_K23)                      /* (3/10)(3 pi^2)^{2/3}, Eq. (tauTFdefn) */
#define OF_CS (1.0 / (4.0 * OF_K23))               /* s^2 = |grad n|^2 OF_CS / n^{8/3} */

template <typename T>
OF_HD FsOut<T> fs_point(const FuncParams &fp, const T *__restrict__ tab, T temp, T n, T g2)
{
    FsOut<T> o;
    T y = inv_cbrt(n);                                  // n^{-1/3}
    o.y13 = y;
    T y2 = y * y;
    T c13 = n * y2;                                     // n^{1/3}
    T n23 = c13 * c13;
    T rn = y2 * y;                                      // 1/n
    T tau0 = T(OF_CTF) * n * n23;                       // Eq. (tauTFdefn)
    T dtau0 = T(5.0 / 3.0 * OF_CTF) * n23;
    T t = T(2.0 / OF_K23) * temp * y2;                  // Eq. (tred)
    T dtdn = T(-2.0 / 3.0) * t * rn;
    T tf[8];
    if (fp.kind == 0) {                                 // ftTF: f = tau0 kappa, kappa = xi - zeta
        tfunc_eval<T, 2>(tab, t, tf);
        T xi = tf[0], ze = tf[1], dxi = tf[4], dze = tf[5];
        o.f = tau0 * (xi - ze);
        o.ts = tau0 * ze;
        o.dfdn = dtau0 * (xi - ze) + tau0 * (dxi - dze) * dtdn;   // Eq. (vTF)
        o.wc = T(0);
        return o;
    }
    tfunc_eval<T>(tab, t, tf);
    T xi = tf[0], ze = tf[1], A = tf[2], B = tf[3];
    T dxi = tf[4], dze = tf[5], dA = tf[6], dB = tf[7];
    // s^2 = |grad n|^2 / (4 (3 pi^2)^{2/3} n^{8/3})  (Eq. (s_0defn))
    T rn43 = rn * y;
    T s2 = (g2 * rn43) * rn43 * T(OF_CS);               // ordered so n^{-8/3} never forms alone
    T xt = s2 * A, xs = s2 * B;                          // s_tau^2, s_sigma^2 (Eq. (s_s))
    T Ft, dFt, Fsg, dFsg;
    enhance<T>(fp, xt, Ft, dFt);
    enhance<T>(fp, xs, Fsg, dFsg);
    T Fs = T(2) - Fsg, dFs = -dFsg;                      // F_sigma = 2 - F_tau(s_sigma)
    T kin = tau0 * xi, ent = tau0 * ze;
    o.f = kin * Ft - ent * Fs;                           // Eq. (FGGA)
    o.ts = ent * Fs;
    T e83 = T(-8.0 / 3.0) * rn;
    // Eq. (vftGGA), first two lines (every sigma term carries the minus sign of Eq. (FGGA))
    o.dfdn = dtau0 * (xi * Ft - ze * Fs) + tau0 * dtdn * (dxi * Ft - dze * Fs)
             + kin * dFt * (e83 * xt + s2 * dA * dtdn)
             - ent * dFs * (e83 * xs + s2 * dB * dtdn);
    // last line: W = [tau0 xi F_tau' A - tau0 zeta F_sigma' B] d s^2/d grad n
    o.wc = ((kin * dFt * A - ent * dFs * B) * rn43) * rn43 * T(2 * OF_CS);
    return o;
}

// Perdew-Zunger 1981 unpolarised LDA: eps_xc and v_xc = eps_xc - (r_s/3) d eps_xc/d r_s.
// gamma, beta1, beta2, A, B as published; C and D are fixed by continuity of
// eps_c and its r_s derivative at r_s = 1 (the published rounded C, D leave a
// small jump there).
constexpr double kPzDen = 1.0 + 1.0529 + 0.3334;
constexpr double kPzD = -0.1423 / kPzDen + 0.048;                                // B + D = eps_pade(1)
constexpr double kPzC = 0.1423 * (0.5 * 1.0529 + 0.3334) / (kPzDen * kPzDen) - 0.0311 - kPzD;

// y = n^{-1/3} as computed by the caller.
template <typename T>
OF_HD void pz81_point(T n, T y, T &eps, T &v)
{
    T rs = T(0.62035049089940001667) * y;              // (3/(4 pi n))^{1/3}
    T ex = T(-0.73855876638202240587) * n * y * y;     // -(3/4)(3/pi)^{1/3} n^{1/3}
    T ec, vc;
    if (rs >= T(1)) {
        T sq = sqrt(rs);
        T den = T(1) / (T(1) + T(1.0529) * sq + T(0.3334) * rs);
        ec = T(-0.1423) * den;
        vc = ec * (T(1) + T(7.0 / 6.0 * 1.0529) * sq + T(4.0 / 3.0 * 0.3334) * rs) * den;
    } else {
        T lr = log(rs);
        ec = T(0.0311) * lr + T(-0.048) + T(kPzC) * rs * lr + T(kPzD) * rs;
        vc = T(0.0311) * lr + T(-0.048 - 0.0311 / 3.0) + T(2.0 / 3.0 * kPzC) * rs * lr
             + T((2.0 * kPzD - kPzC) / 3.0) * rs;
    }
    eps = ex + ec;
    v = T(4.0 / 3.0) * ex + vc;
}

template <typename T>
OF_HD void pz81_point(T n, T &eps, T &v)
{
    pz81_point<T>(n, inv_cbrt(n), eps, v);
}

// ---------------------------------------------------------------------------
// The same pointwise functional in double-float arithmetic (ffmath.cuh) for
// the FP64 path's double-float kernels: every intermediate is a double-float,
// so the result agrees with the binary64 routines above to about 1e-13 of the
// size of its terms while running on the FP32 units.  Outside the domain
// below (and in the Sommerfeld and classical branches of the temperature
// functions) pw_core_f2 returns false and the caller uses binary64.  The
// split table (hi, lo per coefficient) follows the binary64 one.

template <typename T> struct PwOut {
    T f, ts, dfdn, wc, eps, vxc;
};

constexpr double kPwNmin = 1e-18, kPwNmax = 1e18, kPwS2max = 1e10;

#ifndef OFDFT_TF_UNROLL
#define OFDFT_TF_UNROLL 4
#endif
// functions evaluated side by side: fully unrolled, the table values stay
// in registers (a runtime-indexed out[] would live in local memory)
constexpr int kTfUnroll = OFDFT_TF_UNROLL;
#ifndef OFDFT_HORNER_UNROLL
#define OFDFT_HORNER_UNROLL 2
#endif
constexpr int kHornerUnroll = OFDFT_HORNER_UNROLL;   // Horner steps unrolled (code size against loop overhead)

// Horner evaluation of a table polynomial c[0..deg] at the binary32 panel
// variable uh, with its derivative dp and half its second derivative d2:
// the terms of degree >= split in binary32 (their sum, times u^split, is
// below 2^-24 of the polynomial's smallest value on every panel of the
// table, so binary32 rounding there stays below the double-float
// rounding), the rest in double-float.  A split of deg runs every step in
// double-float.
OF_HD void horner_split_f2(const ff::f2 *__restrict__ c, int deg, int split, float uh, ff::f2 &p, ff::f2 &dp,
                           float &d2)
{
    d2 = 0.0f;
    int j = deg - 1;
    if (split < deg) {
        float pf = c[deg].hi, dpf = 0.0f;
#pragma unroll kHornerUnroll
        for (; j >= split; --j) {
            d2 = d2 * uh + dpf;
            dpf = dpf * uh + pf;
            pf = pf * uh + c[j].hi;
        }
        p = {pf, 0.0f};
        dp = {dpf, 0.0f};
    } else {
        p = c[deg];
        dp = {0.0f, 0.0f};
    }
#pragma unroll kHornerUnroll
    for (; j >= 0; --j) {
        d2 = d2 * uh + dp.hi;
        dp = ff::fma_step(dp, uh, p);
        p = ff::fma_step(p, uh, c[j]);
    }
}

// Degree from which the temperature table's terms are summed in binary32,
// per function (xi, zeta, A, B): the largest tails of the fitted
// polynomials, over every panel and relative to the polynomial's smallest
// value there, are 3.3e-9 (xi, degree 7 up) and 2.9e-8 (A, degree 8 up).
// zeta comes close to zero inside some panels, but it enters only beside
// xi (f = tau0 xi F_tau - tau0 zeta F_sigma): its tail from degree 7 up is
// 5.1e-9 of the panel's largest |xi|.  B keeps every term in double-float
// (its monomial coefficients do not decay on the low-t panels).  Against the all-double-float sums the pointwise outputs
// differ by less than their own double-float rounding (host sweep over
// every panel, 1e-16 to 1e6 bohr^-3 at 1e4 K and 1e6 K).
constexpr int kTfSplitXi = 7, kTfSplitZeta = 7, kTfSplitA = 8;
// The enhancement table of G: tail 1.3e-8 from degree 5 up.
constexpr int kEnSplit = 5;

// Table polynomials with a double-float table (same layout as tfunc_eval's).
// The panel variable u = uh + ul: uh is exact in binary32 and the Horner
// sums run with it; ul (below 5e-7) enters through the first and second
// derivatives.
template <int NF>
OF_HD void tfunc_eval_f2(const ff::f2 *__restrict__ tab, ff::f2 t, ff::f2 out[8])
{
    int e;
    float inv2e;
    const float m = split_pow2(t.hi, e, inv2e);
    const int sub = (int)((m - 1.0f) * 4.0f);
    const float uh = 8.0f * (m - 1.0f) - (float)(2 * sub + 1);
    const float ul = 8.0f * t.lo * inv2e;
    const float dudt = 8.0f * inv2e;
    const ff::f2 *c = tab + ((size_t)((e - kTfEmin) * kTfSub + sub) * kTfFuncs) * kTfNc;
#pragma unroll kTfUnroll
    for (int q = 0; q < NF; ++q) {
        ff::f2 p, dp;
        float d2;   // half the second derivative
        horner_split_f2(c + q * kTfNc, kTfDeg, q == 0 ? kTfSplitXi : (q == 1 ? kTfSplitZeta : (q == 2 ? kTfSplitA : kTfDeg)), uh, p, dp, d2);
        p = ff::add(p, dp.hi * ul);
        dp = ff::add(dp, 2.0f * d2 * ul);
        out[q] = p;
        out[4 + q] = ff::scale(dp, dudt);
    }
}

// Enhancement factor F(x) and dF/dx in double-float (forms as in enhance).
FF_CALL void enhance_f2(const FuncParams &fp, ff::f2 x, ff::f2 &F, ff::f2 &dF)
{
    using namespace ff;
    if (fp.kind == 1) {                                     // SGA form
        const f2 p0 = from_double(fp.p0);
        F = add(mul(x, p0), 1.0f);
        dF = p0;
    } else if (fp.kind == 3) {                              // KST2 form
        const f2 p0 = from_double(fp.p0), p1 = from_double(fp.p1);
        f2 den = recip(add(mul(x, p1), 1.0f));
        F = add(mul(mul(x, p0), den), 1.0f);
        dF = mul(p0, mul(den, den));
    } else {                                                // VT84F, m = 8, n = 4
        const f2 mu = FFC(2.778), al = FFC(1.2965);
        if (x.hi <= 1e-15f) {                               // F = 1 + O(x)
            F = {1.0f, 0.0f};
            dF = FFC(-2.778 + 1.2965 + 5.0 / 3.0);
            return;
        }
        const f2 ax = mul(x, al);
        const f2 e1 = exp(neg(ax));                         // e^(-al x)
        const f2 x2 = mul(x, x);
        const f2 em = neg(expm1_neg(neg(mul(x2, al))));     // 1 - e^(-al x^2)
        const f2 mx = mul(x, mu);
        const f2 q = add(mx, 1.0f);                         // 1 + mu x
        const f2 inv = recip(mul(x, q));
        const f2 rx = mul(q, inv);                          // 1/x
        const f2 den = mul(x, inv);                         // 1/(1 + mu x)
        // F = 1 - mu x e1 den + em (rx - 1) + (5/3) x
        f2 Fv = add(neg(mul(mul(mx, e1), den)), 1.0f);
        Fv = add(Fv, mul(em, add(rx, -1.0f)));
        F = add(Fv, mul(x, FFC(5.0 / 3.0)));
        // dF = -mu e1 (1 - al x - al mu x^2) den^2 + 2 al (1 - em)(1 - x) - em rx^2 + 5/3
        const f2 poly = add(neg(add(ax, mul(mul(x2, al), mu))), 1.0f);
        f2 d = neg(mul(mul(mul(mu, e1), poly), mul(den, den)));
        d = add(d, mul(mul(al, add(neg(em), 1.0f)), scale(add(neg(x), 1.0f), 2.0f)));
        d = sub(d, mul(em, mul(rx, rx)));
        dF = add(d, FFC(5.0 / 3.0));
    }
}

// VT84F F(x) and dF/dx in double-float from the enhancement table etab of
// G = (F - 1)/x (kEnSize pairs): F = 1 + x G, dF = G + x G' with G' the
// polynomial's derivative, so the potential is the exact derivative of the
// tabulated energy; x < 2^-20: the cubic series (the next terms are below
// 1e-16 in F and dF), x >= 64: F = 5x/3 + 1/x.
OF_HD void enhance_vt84f_tab(const ff::f2 *__restrict__ etab, ff::f2 x, ff::f2 &F, ff::f2 &dF)
{
    using namespace ff;
    if (x.hi < 9.5367431640625e-07f) {
        // series of Eq. (VT84F): c1 = alpha - mu + 5/3, c2 = mu (alpha + mu) - alpha,
        // c3 = -mu (alpha^2/2 + alpha mu + mu^2) - alpha^2/2 (the x^3 term matters
        // for dF at the 1e-12 level)
        constexpr double mu = 2.778, al = 1.2965;
        constexpr double c1 = al - mu + 5.0 / 3.0, c2 = mu * (al + mu) - al;
        constexpr double c3 = -mu * (0.5 * al * al + al * mu + mu * mu) - 0.5 * al * al;
        F = add(mul(x, add(mul(x, add(mul(x, FFC(c3)), FFC(c2))), FFC(c1))), 1.0f);
        dF = add(mul(x, add(mul(x, FFC(3.0 * c3)), FFC(2.0 * c2))), FFC(c1));
        return;
    }
    if (x.hi >= 64.0f) {
        const f2 r = recip(x);
        F = add(mul(x, FFC(5.0 / 3.0)), r);
        dF = sub(FFC(5.0 / 3.0), mul(r, r));
        return;
    }
    int e;
    float inv2e;
    const float m = split_pow2(x.hi, e, inv2e);
    const int sub = (int)((m - 1.0f) * (float)kEnSub);
    const float uh = (float)(2 * kEnSub) * (m - 1.0f) - (float)(2 * sub + 1);
    const float ul = (float)(2 * kEnSub) * x.lo * inv2e;
    const float dudx = (float)(2 * kEnSub) * inv2e;
    const f2 *c = etab + (size_t)((e - kEnEmin) * kEnSub + sub) * kEnNc;
    f2 p, dp;
    float d2;   // half the second derivative
    horner_split_f2(c, kEnDeg, kEnSplit, uh, p, dp, d2);
    const f2 G = add(p, dp.hi * ul);
    const f2 dG = scale(add(dp, 2.0f * d2 * ul), dudx);
    F = add(mul(x, G), 1.0f);
    dF = add(G, mul(x, dG));
}

// PZ81 (same branches and constants as pz81_point) from n, n^(1/3) and
// y = n^(-1/3) in double-float.
OF_HD void pz81_f2(ff::f2 c13, ff::f2 y, ff::f2 &eps, ff::f2 &v)
{
    using namespace ff;
    const f2 rs = mul(y, FFC(0.62035049089940001667));
    const f2 ex = mul(c13, FFC(-0.73855876638202240587));
    f2 ec, vc;
    if (rs.hi >= 1.0f) {
        const f2 sq = sqrt(rs);
        const f2 den = recip(add(add(mul(sq, FFC(1.0529)), mul(rs, FFC(0.3334))), 1.0f));
        ec = mul(den, FFC(-0.1423));
        const f2 num = add(add(mul(sq, FFC(7.0 / 6.0 * 1.0529)), mul(rs, FFC(4.0 / 3.0 * 0.3334))), 1.0f);
        vc = mul(mul(ec, num), den);
    } else {
        const f2 lr = log(rs);
        const f2 rlr = mul(rs, lr);
        ec = add(add(mul(lr, FFC(0.0311)), FFC(-0.048)), add(mul(rlr, FFC(kPzC)), mul(rs, FFC(kPzD))));
        vc = add(add(mul(lr, FFC(0.0311)), FFC(-0.048 - 0.0311 / 3.0)),
                 add(mul(rlr, FFC(2.0 / 3.0 * kPzC)), mul(rs, FFC((2.0 * kPzD - kPzC) / 3.0))));
    }
    eps = add(ex, ec);
    v = add(mul(ex, FFC(4.0 / 3.0)), vc);
}

// Double-float outputs of the pointwise functional at one point.
struct PwF2 {
    ff::f2 f, ts, dfdn, eps, vxc;
    ff::f2 w[3];    // W = d f_s / d(grad n), by component
};

// f_s, its derivatives and (xc != 0) PZ81 at one point from n and the
// gradient components gr[3] in double-float; false when the point is
// outside the double-float domain (s^2 is formed from (grad n) n^(-4/3), so
// an s^2 past kPwS2max, or one that overflows, also returns false).
// tcoef = 2 k_B T / (3 pi^2)^(2/3).
OF_HD bool pw_core_f2(const FuncParams &fp, const ff::f2 *__restrict__ tab, ff::f2 tcoef, ff::f2 n,
                      const ff::f2 *gr, int xc, PwF2 &o)
{
    using namespace ff;
    if (!(n.hi >= (float)kPwNmin && n.hi <= (float)kPwNmax)) return false;
    const f2 y = rcbrt(n);                                   // n^(-1/3)
    const f2 y2 = mul(y, y);
    const f2 t = mul(tcoef, y2);                             // Eq. (tred)
    if (!(t.hi >= 9.5367431640625e-07f && t.hi < 17179869184.0f)) return false;
    const f2 c13 = mul(n, y2);                               // n^(1/3)
    const f2 n23 = mul(c13, c13);
    const f2 rn = mul(y2, y);                                // 1/n
    const f2 tau0 = mul(mul(n, n23), FFC(OF_CTF));           // Eq. (tauTFdefn)
    const f2 dtau0 = mul(n23, FFC(5.0 / 3.0 * OF_CTF));
    const f2 dtdn = mul(mul(t, rn), FFC(-2.0 / 3.0));
    f2 tf[8];
    if (fp.kind == 0) {                                      // ftTF
        tfunc_eval_f2<2>(tab, t, tf);
        const f2 kap = sub(tf[0], tf[1]);
        o.f = mul(tau0, kap);
        o.ts = mul(tau0, tf[1]);
        o.dfdn = add(mul(dtau0, kap), mul(mul(tau0, sub(tf[4], tf[5])), dtdn));   // Eq. (vTF)
        o.w[0] = o.w[1] = o.w[2] = f2(0.0f, 0.0f);
    } else {
        const f2 rn43 = mul(y2, y2);                         // n^(-4/3)
        const f2 q0 = mul(gr[0], rn43), q1 = mul(gr[1], rn43), q2 = mul(gr[2], rn43);
        const f2 s2 = mul(add(add(mul(q0, q0), mul(q1, q1)), mul(q2, q2)), FFC(OF_CS));   // Eq. (s_0defn)
        if (!(s2.hi <= (float)kPwS2max)) return false;
        tfunc_eval_f2<4>(tab, t, tf);
        const f2 xi = tf[0], ze = tf[1], A = tf[2], B = tf[3];
        const f2 dxi = tf[4], dze = tf[5], dA = tf[6], dB = tf[7];
        const f2 xt = mul(s2, A), xs = mul(s2, B);           // Eq. (s_s)
        f2 Ft, dFt, Fsg, dFsg;
        if (fp.kind == 2) {                                  // VT84F: the enhancement table
            const f2 *etab = tab + kTfSize;
            enhance_vt84f_tab(etab, xt, Ft, dFt);
            enhance_vt84f_tab(etab, xs, Fsg, dFsg);
        } else {
            enhance_f2(fp, xt, Ft, dFt);
            enhance_f2(fp, xs, Fsg, dFsg);
        }
        const f2 Fs = add(neg(Fsg), 2.0f), dFs = neg(dFsg); // F_sigma = 2 - F_tau(s_sigma)
        const f2 kin = mul(tau0, xi), ent = mul(tau0, ze);
        o.f = sub(mul(kin, Ft), mul(ent, Fs));              // Eq. (FGGA)
        o.ts = mul(ent, Fs);
        const f2 e83 = mul(rn, FFC(-8.0 / 3.0));
        const f2 s2dt = mul(s2, dtdn);
        // Eq. (vftGGA), first two lines
        f2 d = mul(dtau0, sub(mul(xi, Ft), mul(ze, Fs)));
        d = add(d, mul(mul(tau0, dtdn), sub(mul(dxi, Ft), mul(dze, Fs))));
        d = add(d, mul(mul(kin, dFt), add(mul(e83, xt), mul(s2dt, dA))));
        d = sub(d, mul(mul(ent, dFs), add(mul(e83, xs), mul(s2dt, dB))));
        o.dfdn = d;
        // last line: W = [tau0 xi F_tau' A - tau0 zeta F_sigma' B] d s^2 / d grad n
        const f2 wpre = sub(mul(mul(kin, dFt), A), mul(mul(ent, dFs), B));
        const f2 wr = mul(mul(wpre, rn43), FFC(2.0 * OF_CS));
        for (int a = 0; a < 3; ++a) o.w[a] = mul(wr, mul(gr[a], rn43));
    }
    if (xc) {
        pz81_f2(c13, y, o.eps, o.vxc);
    } else {
        o.eps = f2(0.0f, 0.0f);
        o.vxc = f2(0.0f, 0.0f);
    }
    return true;
}

// The routines of the precision T (binary64 or binary32) with the same output.
template <typename T>
OF_HD PwOut<T> pw_point_native(const FuncParams &fp, const T *__restrict__ tab, T temp, T n, T g2, int xc)
{
    FsOut<T> s = fs_point<T>(fp, tab, temp, n, g2);
    PwOut<T> o;
    o.f = s.f;
    o.ts = s.ts;
    o.dfdn = s.dfdn;
    o.wc = s.wc;
    o.eps = T(0);
    o.vxc = T(0);
    if (xc) pz81_point<T>(n, s.y13, o.eps, o.vxc);
    return o;
}


// Double-float table written from the binary64 one (hi, lo per coefficient).
inline void tfunc_table_split(const double *tab, float *out, int count = kTfSize)
{
    for (int i = 0; i < count; ++i) {
        ff::f2 c = ff::from_double(tab[i]);
        out[2 * i] = c.hi;
        out[2 * i + 1] = c.lo;
    }
}

// The FP64 field sets' tables in dst[kDdTabSize]: the binary64 temperature
// table, its double-float split, the double-float VT84F enhancement table
// (the split temperature table and the enhancement table are contiguous,
// as pw_core_f2 reads them).
inline void dd_tables_fill(const double *ttab, double *dst)
{
    for (int i = 0; i < kTfSize; ++i) dst[i] = ttab[i];
    tfunc_table_split(ttab, reinterpret_cast<float *>(dst + kTfSize));
    double etab[kEnSize];
    enh_table_fill(etab);
    tfunc_table_split(etab, reinterpret_cast<float *>(dst + 2 * kTfSize), kEnSize);
}

}  // namespace ofdft
