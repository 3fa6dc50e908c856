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

}  // namespace ofdft
