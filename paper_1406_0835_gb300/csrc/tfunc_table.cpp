// Tabulated temperature functions of finite-T orbital-free DFT.
//
// For the reduced temperature t = T/T_F of Eq. (tred) the kernels need
//   xi(t)   = kappa - t kappa'                  (Eq. (xizeta))
//   zeta(t) = -t kappa'
//   A(t)    = (h~ - t h~')/xi,  B(t) = t h~'/zeta   (s_tau^2 = s^2 A, s_sigma^2 = s^2 B, Eq. (s_s))
// and their t-derivatives.  kappa is the ideal-gas free energy per particle
// over tau0 (footnote a of Table I: kappa = (5/3) t f(y)); h~ is Perrot's
// finite-T gradient coefficient, read here as the q^2 coefficient of the
// finite-T Lindhard function: h~ = 6 I_{1/2} I'_{-1/2} / I_{-1/2}^2.
//
// This file builds, once per process, piecewise polynomial fits of xi, zeta,
// A, B in t (and, for the double-float kernels, of the VT84F enhancement
// factor in x = s^2, enh_table_fill): 4 panels per octave of t over [2^-20, 2^34), degree 10 in the
// panel variable u in [-1, 1).  The kernels differentiate the polynomials, so
// the potential is the exact derivative of the tabulated energy.
//
// Values at the nodes come from Fermi-Dirac integrals computed here:
// composite 24-point Gauss-Legendre quadrature in u = sqrt(x) for eta < 40,
// the Sommerfeld series with zeta(2k) from closed forms and direct sums for
// eta >= 40, and xi = (5/2) t^{5/2} I_{3/2} (the ideal-gas identity
// u = (3/2) P written with tau0 = (3/5) n T_F).
#include <cmath>
#include <mutex>
#include <vector>

#include "ofdft_internal.h"

namespace ofdft {
namespace {

const double kPi = 3.14159265358979323846;

struct GL24 {
    double x[24], w[24];
    GL24()
    {
        const int n = 24;
        for (int i = 0; i < n; ++i) {
            // Newton on the Legendre polynomial from the Tricomi initial guess
            double z = std::cos(kPi * (4.0 * i + 3.0) / (4.0 * n + 2.0));
            double dp = 1.0;
            for (int it = 0; it < 60; ++it) {
                double p0 = 1.0, p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                double step = p1 / dp;
                z -= step;
                if (std::fabs(step) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

// moments: I_{-1/2}, I_{1/2}, I_{3/2}, I'_{-1/2}, I''_{-1/2}, I'''_{-1/2}
void moments_quadrature(double eta, double m[6])
{
    static const GL24 gl;
    for (int k = 0; k < 6; ++k) m[k] = 0.0;
    double U = std::sqrt((eta > 0.0 ? eta : 0.0) + 48.0);
    const double hu = 0.25;
    int npan = (int)std::ceil(U / hu);
    for (int p = 0; p < npan; ++p) {
        double a = p * hu, b = (p + 1) * hu;
        double c = 0.5 * (a + b), h = 0.5 * (b - a);
        for (int i = 0; i < 24; ++i) {
            double u = c + h * gl.x[i];
            double w = 2.0 * h * gl.w[i];  // dx = 2 u du; the u is folded below
            double y = u * u - eta;
            double f, fc;
            if (y > 0) {
                double e = std::exp(-y);
                f = e / (1.0 + e);
                fc = 1.0 / (1.0 + e);
            } else {
                double e = std::exp(y);
                f = 1.0 / (1.0 + e);
                fc = e / (1.0 + e);
            }
            double p1 = f * fc;
            double u2 = u * u;
            m[0] += w * f;                    // x^{-1/2} dx = 2 du
            m[1] += w * u2 * f;               // x^{1/2} dx = 2 u^2 du
            m[2] += w * u2 * u2 * f;          // x^{3/2} dx = 2 u^4 du
            m[3] += w * p1;
            m[4] += w * p1 * (1.0 - 2.0 * f);
            m[5] += w * p1 * (1.0 - 6.0 * p1);
        }
    }
}

// Dirichlet eta(2k) = (1 - 2^{1-2k}) zeta(2k).
double dirichlet_eta_even(int k)
{
    double z;
    switch (k) {
    case 1: z = kPi * kPi / 6.0; break;
    case 2: z = std::pow(kPi, 4) / 90.0; break;
    case 3: z = std::pow(kPi, 6) / 945.0; break;
    case 4: z = std::pow(kPi, 8) / 9450.0; break;
    default: {
        z = 0.0;   // n^{-2k} for k >= 5: terms past n = 60 are below 1e-35
        for (int n = 60; n >= 1; --n) z += std::pow((double)n, -2.0 * k);
    }
    }
    return (1.0 - std::pow(2.0, 1.0 - 2.0 * k)) * z;
}

// Complete FD integral F_j(eta) (= I_j / Gamma(j+1)) for eta >= 40 by the
// Sommerfeld series sum_k 2 eta_D(2k) eta^{j+1-2k} / Gamma(j+2-2k), eta_D(0) = 1/2.
double fd_complete_series(double j, double eta)
{
    static double coef[40];
    static std::once_flag once;
    std::call_once(once, [] {
        coef[0] = 0.5;
        for (int k = 1; k < 40; ++k) coef[k] = dirichlet_eta_even(k);
    });
    double inv_gamma = 1.0 / std::tgamma(j + 2.0);
    double pw = std::pow(eta, j + 1.0);
    double sum = 2.0 * coef[0] * pw * inv_gamma;
    double last = std::fabs(sum);
    for (int k = 1; k < 40; ++k) {
        double z = j + 2.0 - 2.0 * k;          // Gamma(z+2) = (z+1) z Gamma(z)
        inv_gamma *= z * (z + 1.0);
        pw /= eta * eta;
        double term = 2.0 * coef[k] * pw * inv_gamma;
        if (std::fabs(term) >= last) break;
        sum += term;
        last = std::fabs(term);
        if (last < 1e-19 * std::fabs(sum)) break;
    }
    return sum;
}

void moments(double eta, double m[6])
{
    if (eta < 40.0) {
        moments_quadrature(eta, m);
        return;
    }
    const double sp = std::sqrt(kPi);
    m[0] = sp * fd_complete_series(-0.5, eta);
    m[1] = 0.5 * sp * fd_complete_series(0.5, eta);
    m[2] = 0.75 * sp * fd_complete_series(1.5, eta);
    m[3] = sp * fd_complete_series(-1.5, eta);
    m[4] = sp * fd_complete_series(-2.5, eta);
    m[5] = sp * fd_complete_series(-3.5, eta);
}

// eta with I_{1/2}(eta) = y by Newton in eta, bisection once bracketed.
double solve_eta(double y)
{
    double eta = (y < 1.5) ? std::log(y / 0.886226925452758014) : std::pow(1.5 * y, 2.0 / 3.0);
    double lo = -1e300, hi = 1e300, m[6];
    for (int it = 0; it < 300; ++it) {
        moments(eta, m);
        double r = m[1] - y;
        if (r > 0) hi = eta < hi ? eta : hi;
        else lo = eta > lo ? eta : lo;
        double step = r / (0.5 * m[0]);
        if (std::fabs(step) <= 1e-15 * (std::fabs(eta) > 1.0 ? std::fabs(eta) : 1.0)) {
            eta -= step;
            break;
        }
        double nxt = eta - step;
        if (lo > -1e299 && hi < 1e299 && (nxt <= lo || nxt >= hi)) nxt = 0.5 * (lo + hi);
        double cap = std::fabs(eta) > 8.0 ? std::fabs(eta) : 8.0;
        if (nxt > eta + cap) nxt = eta + cap;
        if (nxt < eta - cap) nxt = eta - cap;
        eta = nxt;
    }
    return eta;
}

// xi, zeta, A, B at t.
void tfuncs(double t, double f[4])
{
    double y = (2.0 / 3.0) * std::pow(t, -1.5);
    double eta = solve_eta(y);
    double m[6];
    moments(eta, m);
    double Im = m[0], Ih = m[1], I3 = m[2], Ip = m[3], Ipp = m[4];
    double t52 = std::pow(t, 2.5);
    double xi = 2.5 * t52 * I3;
    double zeta = (25.0 / 6.0) * t52 * I3 - (5.0 / 3.0) * t * eta;
    // h~ = 6 a b / c^2 with a = I_{1/2}, b = I'_{-1/2}, c = I_{-1/2};
    // dh~/deta = 6 [(a'b + a b') c - 2 a b c'] / c^3, a' = c/2, c' = b.
    double dh_deta = 6.0 * ((0.5 * Im * Ip + Ih * Ipp) * Im - 2.0 * Ih * Ip * Ip) / (Im * Im * Im);
    double h = 6.0 * Ih * Ip / (Im * Im);
    double deta_dt = -2.0 / (t52 * Im);
    double th1 = t * dh_deta * deta_dt;   // t h~'
    f[0] = xi;
    f[1] = zeta;
    f[2] = (h - th1) / xi;
    f[3] = th1 / zeta;
}

}  // namespace

// Fill tab[kTfSize] (no allocation: node values and fits live on the stack).
void tfunc_table_fill(double *tab)
{
    const int d = kTfDeg, nc = kTfNc;
    for (int i = 0; i < kTfSize; ++i) tab[i] = 0.0;
    double un[nc];
    for (int k = 0; k < nc; ++k) un[k] = std::cos(kPi * (k + 0.5) / nc);
    // monomial coefficients of Chebyshev polynomials T_0..T_d
    double Tm[nc][nc];
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j) Tm[i][j] = 0.0;
    Tm[0][0] = 1.0;
    if (d >= 1) Tm[1][1] = 1.0;
    for (int i = 2; i <= d; ++i)
        for (int j = 0; j <= i; ++j)
            Tm[i][j] = (j > 0 ? 2.0 * Tm[i - 1][j - 1] : 0.0) - Tm[i - 2][j];
    for (int e = kTfEmin; e < kTfEmax; ++e) {
        for (int s = 0; s < kTfSub; ++s) {
            double vals[kTfFuncs][nc];
            for (int k = 0; k < nc; ++k) {
                double t = std::ldexp(1.0 + 0.25 * s + 0.125 * (un[k] + 1.0), e);
                double f[4];
                tfuncs(t, f);
                for (int q = 0; q < kTfFuncs; ++q) vals[q][k] = f[q];
            }
            int panel = (e - kTfEmin) * kTfSub + s;
            for (int q = 0; q < kTfFuncs; ++q) {
                double cheb[nc];
                for (int j = 0; j < nc; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < nc; ++k) acc += vals[q][k] * std::cos(kPi * j * (k + 0.5) / nc);
                    cheb[j] = (j == 0 ? 1.0 : 2.0) * acc / nc;
                }
                double *out = &tab[((size_t)panel * kTfFuncs + q) * nc];
                for (int j = 0; j < nc; ++j) {
                    double a = 0.0;
                    for (int i = j; i < nc; ++i) a += cheb[i] * Tm[i][j];
                    out[j] = a;
                }
            }
        }
    }
}

// VT84F (Eq. (VT84F) with m = 8, n = 4, written in x = s^2) through
// G(x) = (F(x) - 1)/x, which stays of order one as x -> 0 (so the fitted
// slope keeps its relative accuracy there):
//   G = -mu e^(-alpha x)/(1 + mu x) + (1 - e^(-alpha x^2))/x^2
//       - (1 - e^(-alpha x^2))/x + 5/3,
// evaluated in long double and fitted per panel: Chebyshev interpolation
// at kEnNc nodes, then monomial coefficients in the panel variable u
// (x = 2^e (1 + (sub + (u + 1)/2)/kEnSub)).
void enh_table_fill(double *tab)
{
    // the fit runs in long double: the slope of G on a narrow panel is small
    // next to G, and binary64 rounding of the interpolation would swamp it
    const long double mu = 2.778L, al = 1.2965L, pi = 3.14159265358979323846264338327950288L;
    const int d = kEnDeg, nc = kEnNc;
    long double un[nc];
    for (int k = 0; k < nc; ++k) un[k] = std::cos(pi * (k + 0.5L) / nc);
    long double Tm[nc][nc];
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j) Tm[i][j] = 0.0L;
    Tm[0][0] = 1.0L;
    Tm[1][1] = 1.0L;
    for (int i = 2; i <= d; ++i)
        for (int j = 0; j <= i; ++j)
            Tm[i][j] = (j > 0 ? 2.0L * Tm[i - 1][j - 1] : 0.0L) - Tm[i - 2][j];
    for (int e = kEnEmin; e < kEnEmax; ++e) {
        for (int sub = 0; sub < kEnSub; ++sub) {
            long double vals[nc];
            for (int k = 0; k < nc; ++k) {
                const long double x = std::ldexp(1.0L + (sub + 0.5L * (un[k] + 1.0L)) / kEnSub, e);
                const long double e1 = std::exp(-al * x);
                const long double em = -std::expm1(-al * x * x);     // 1 - e^(-alpha x^2)
                vals[k] = -mu * e1 / (1.0L + mu * x) + em / (x * x) - em / x + 5.0L / 3.0L;
            }
            long double cheb[nc];
            for (int j = 0; j < nc; ++j) {
                long double acc = 0.0L;
                for (int k = 0; k < nc; ++k) acc += vals[k] * std::cos(pi * j * (k + 0.5L) / nc);
                cheb[j] = (j == 0 ? 1.0L : 2.0L) * acc / nc;
            }
            double *out = &tab[(size_t)((e - kEnEmin) * kEnSub + sub) * nc];
            for (int j = 0; j < nc; ++j) {
                long double a = 0.0L;
                for (int i = j; i < nc; ++i) a += cheb[i] * Tm[i][j];
                out[j] = (double)a;
            }
        }
    }
}

namespace {

std::vector<double> build_table()
{
    std::vector<double> tab((size_t)kTfSize, 0.0);
    tfunc_table_fill(tab.data());
    return tab;
}

}  // namespace

const std::vector<double> &tfunc_table_host()
{
    static std::vector<double> tab;
    static std::once_flag once;
    std::call_once(once, [] { tab = build_table(); });
    return tab;
}

}  // namespace ofdft
