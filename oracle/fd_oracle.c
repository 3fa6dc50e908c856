/*
 * Oracle (TEST INFRASTRUCTURE ONLY): Fermi-Dirac integrals and the
 * temperature functions kappa(t) and h~(t) of finite-temperature
 * orbital-free DFT, in plain FP64 C.
 *
 * Only tests/, __graft_entry__.smoke() and the cpu_baseline leg of bench.py
 * may load this code.  It shares nothing with the CUDA library.
 *
 * What it computes (Sec. III A, Eqs. (tred), (fTF), footnote a of Table I):
 *   I_nu(eta) = int_0^inf x^nu / (1 + exp(x - eta)) dx,  nu = -1/2, 1/2, 3/2,
 *   and the eta-derivatives of I_{-1/2} up to third order, by composite
 *   Gauss-Legendre quadrature (20 nodes per panel).
 *   For a spin-unpolarised ideal Fermi gas n = (sqrt2/pi^2) T^{3/2} I_{1/2},
 *   so the reduced temperature t = T/T_F of Eq. (tred) fixes
 *   y = I_{1/2}(eta) = (2/3) t^{-3/2}; eta is found by safeguarded Newton.
 *   kappa(t) = (5/3) t f(y) with f(y) = eta - (2/3) I_{3/2}/y, the ideal-gas
 *   free energy per particle in units of T (footnote a of Table I).
 *   h~(t) = 6 I_{1/2} I'_{-1/2} / I_{-1/2}^2: the q^2 coefficient of the
 *   finite-T Lindhard response (Perrot's gradient correction, cited at
 *   Eq. (s_s) and in Table I), written so that the SGA of Eq. (SGA-F)
 *   equals ftTF + (1/72) h~ |grad n|^2 / n.  This formula is a reading:
 *   the paper cites h~ without printing it.
 *
 * Quadrature error budget (eta < 40): every panel [a,b] is no wider than
 * the distance from its centre to the nearest singularity of the integrand
 * (the Fermi poles at x = eta +- i pi, the branch point of x^nu at 0), so
 * the 20-point rule converges like rho^-40 with rho >= 4.2, far below 1e-16.
 * For eta >= 40 the Sommerfeld series replaces the quadrature.
 */
#include <math.h>
#include <stddef.h>

#define NGL 20
static double gl_x[NGL], gl_w[NGL];
static int gl_ready = 0;

/* Gauss-Legendre nodes and weights on [-1,1] by Newton on P_NGL. */
static void som_init(void);

static void gl_init(void)
{
    som_init();
    if (gl_ready) return;
    for (int i = 0; i < NGL; ++i) {
        double z = cos(M_PI * (i + 0.75) / (NGL + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= NGL; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = NGL * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        gl_x[i] = z;
        gl_w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
    gl_ready = 1;
}

/* Fermi function f = 1/(1+e^y) and 1-f, both without cancellation. */
static void fermi(double y, double *f, double *fc)
{
    if (y > 0.0) {
        double e = exp(-y);
        *f = e / (1.0 + e);
        *fc = 1.0 / (1.0 + e);
    } else {
        double e = exp(y);
        *f = 1.0 / (1.0 + e);
        *fc = e / (1.0 + e);
    }
}

/*
 * Riemann zeta at s >= 2 by Euler-Maclaurin summation with N = 30 and the
 * Bernoulli terms B2..B10; the first omitted term is below 1e-19.
 */
static double zeta_em(double s)
{
    const int N = 30;
    const double B[5] = {1.0 / 6.0, -1.0 / 30.0, 1.0 / 42.0, -1.0 / 30.0, 5.0 / 66.0};
    double sum = 0.0;
    for (int n = N - 1; n >= 1; --n) sum += pow((double)n, -s);
    double Nn = (double)N;
    sum += pow(Nn, 1.0 - s) / (s - 1.0) + 0.5 * pow(Nn, -s);
    double rise = s, fact = 2.0; /* s(s+1)...(s+2j-2), (2j)! */
    for (int j = 1; j <= 5; ++j) {
        sum += B[j - 1] / fact * rise * pow(Nn, -s - 2.0 * j + 1.0);
        rise *= (s + 2.0 * j - 1.0) * (s + 2.0 * j);
        fact *= (2.0 * j + 1.0) * (2.0 * j + 2.0);
    }
    return sum;
}

/*
 * Complete Fermi-Dirac integral F_j(eta) = I_j(eta)/Gamma(j+1) for eta >= 40
 * by the Sommerfeld expansion
 *   F_j(eta) = sum_k 2 t_2k eta^{j+1-2k} / Gamma(j+2-2k),
 *   t_0 = 1/2, t_2k = (1 - 2^{1-2k}) zeta(2k),
 * summed while the terms decrease.  Its truncation error and the neglected
 * lower-limit term are both of order exp(-eta) <= 4e-18.
 */
#define NSOM 40
static double som_t2k[NSOM];
static int som_ready = 0;

static void som_init(void)
{
    if (som_ready) return;
    for (int k = 1; k < NSOM; ++k)
        som_t2k[k] = (1.0 - pow(2.0, 1.0 - 2.0 * k)) * zeta_em(2.0 * k);
    som_ready = 1;
}

static double fd_sommerfeld(double j, double eta)
{
    double rg = 1.0 / tgamma(j + 2.0); /* 1/Gamma(j+2-2k) at k = 0 */
    double pw = pow(eta, j + 1.0);
    double sum = pw * rg, prev = fabs(sum);
    double ie2 = 1.0 / (eta * eta);
    for (int k = 1; k < NSOM; ++k) {
        double z = j + 2.0 - 2.0 * k; /* 1/Gamma(z) = (z)(z+1)/Gamma(z+2) */
        rg *= z * (z + 1.0);
        pw *= ie2;
        double term = 2.0 * som_t2k[k] * pw * rg;
        if (fabs(term) > prev) break;
        sum += term;
        prev = fabs(term);
        if (prev < 1e-20 * fabs(sum)) break;
    }
    return sum;
}

/*
 * Moments m[0..5] = I_{-1/2}, I_{1/2}, I_{3/2}, dI_{-1/2}/deta,
 * d2I_{-1/2}/deta2, d3I_{-1/2}/deta3.  d^k f(x-eta)/deta^k:
 *   k=1: f(1-f);  k=2: f(1-f)(1-2f);  k=3: f(1-f)(1-6f(1-f)).
 * For eta >= 40 the Sommerfeld series is used instead of quadrature, with
 * dI_{-1/2}/deta = Gamma(1/2) F_{-3/2} and so on (F_j' = F_{j-1}); the
 * quadrature of the sign-changing derivative integrands would lose about
 * eta^k relative digits there.
 * nmom = 2 stops after I_{-1/2}, I_{1/2} (used inside Newton).
 */
static void fd_moments(double eta, double m[6], int nmom)
{
    const double sqpi = 1.77245385090551602730; /* Gamma(1/2) */
    if (eta >= 40.0) {
        m[0] = sqpi * fd_sommerfeld(-0.5, eta);
        m[1] = 0.5 * sqpi * fd_sommerfeld(0.5, eta);
        if (nmom > 2) {
            m[2] = 0.75 * sqpi * fd_sommerfeld(1.5, eta);
            m[3] = sqpi * fd_sommerfeld(-1.5, eta);
            m[4] = sqpi * fd_sommerfeld(-2.5, eta);
            m[5] = sqpi * fd_sommerfeld(-3.5, eta);
        }
        return;
    }
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double xhi = (eta > 0.0 ? eta : 0.0) + 50.0;
    gl_init();
    /* x in [0,1] with x = u^2: x^nu dx = 2 u^{2nu+1} du, smooth in u. */
    for (int i = 0; i < NGL; ++i) {
        double u = 0.5 * (gl_x[i] + 1.0), w = 0.5 * gl_w[i];
        double x = u * u, f, fc;
        fermi(x - eta, &f, &fc);
        double p = f * fc;
        acc[0] += 2.0 * w * f;
        acc[1] += 2.0 * w * x * f;
        if (nmom > 2) {
            acc[2] += 2.0 * w * x * x * f;
            acc[3] += 2.0 * w * p;
            acc[4] += 2.0 * w * p * (fc - f);
            acc[5] += 2.0 * w * p * (1.0 - 6.0 * p);
        }
    }
    double a = 1.0;
    while (a < xhi) {
        double wdt = a < M_PI ? a : M_PI; /* b <= 2a near 0, width <= pi elsewhere */
        double b = a + wdt;
        if (b > xhi) b = xhi;
        double c = 0.5 * (a + b), h = 0.5 * (b - a);
        for (int i = 0; i < NGL; ++i) {
            double x = c + h * gl_x[i], w = h * gl_w[i];
            double f, fc;
            fermi(x - eta, &f, &fc);
            double sx = sqrt(x);
            double wm = w / sx; /* x^{-1/2} dx */
            double p = f * fc;
            acc[0] += wm * f;
            acc[1] += w * sx * f;
            if (nmom > 2) {
                acc[2] += w * x * sx * f;
                acc[3] += wm * p;
                acc[4] += wm * p * (fc - f);
                acc[5] += wm * p * (1.0 - 6.0 * p);
            }
        }
        a = b;
    }
    for (int k = 0; k < 6; ++k) m[k] = acc[k];
}

/* Starting guess for I_{1/2}(eta) = y: two-term classical or Sommerfeld inversion. */
static double eta_guess(double y)
{
    const double g32 = 0.88622692545275801365; /* Gamma(3/2) */
    double u = y / g32;
    if (u < 2.0) return log(u) + u * 0.35355339059327376220; /* + u / 2^{3/2} */
    double e0 = pow(1.5 * y, 2.0 / 3.0);
    double c = 1.0 - M_PI * M_PI / (12.0 * e0 * e0);
    return e0 * (c > 0.5 ? c : 0.5);
}

/* Solve ln I_{1/2}(eta) = ln y by Newton with a bracket (ln I_{1/2} is increasing). */
static double eta_of_y(double y)
{
    double eta = eta_guess(y), lo = -INFINITY, hi = INFINITY;
    double ly = log(y), m[6], prev_step = INFINITY;
    for (int it = 0; it < 200; ++it) {
        fd_moments(eta, m, 2);
        double F = log(m[1]) - ly;
        if (F > 0.0) { if (eta < hi) hi = eta; }
        else { if (eta > lo) lo = eta; }
        double dF = 0.5 * m[0] / m[1]; /* I'_{1/2} = I_{-1/2}/2 */
        double nxt = eta - F / dF;
        /* Stop at the rounding floor of the quadrature (~1e-15 relative in
         * I_{1/2}), or once the step stops shrinking (rounding noise). */
        double step = fabs(nxt - eta);
        double tol = 4e-15 * (fabs(eta) > 1.0 ? fabs(eta) : 1.0);
        if (step <= tol || (step < 1e-12 && step >= 0.5 * prev_step)) {
            eta = nxt;
            break;
        }
        prev_step = step;
        double lim = fabs(eta) > 10.0 ? fabs(eta) : 10.0;
        if (nxt - eta > lim) nxt = eta + lim;
        if (eta - nxt > lim) nxt = eta - lim;
        if (isfinite(lo) && isfinite(hi) && (nxt <= lo || nxt >= hi)) nxt = 0.5 * (lo + hi);
        eta = nxt;
    }
    return eta;
}

/* Public: Fermi-Dirac moments at given eta, out[i*6 + k]. */
int oracle_fd_moments(long n, const double *eta, double *out)
{
    gl_init();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) fd_moments(eta[i], out + 6 * i, 6);
    return 0;
}

/* Public: eta(t) from I_{1/2}(eta) = (2/3) t^{-3/2}. */
int oracle_eta_of_t(long n, const double *t, double *eta)
{
    gl_init();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) eta[i] = eta_of_y((2.0 / 3.0) * pow(t[i], -1.5));
    return 0;
}

/*
 * Public: per reduced temperature t, out[i*7 + k] =
 *   eta, kappa, dkappa/dt, d2kappa/dt2, h~, dh~/dt, d2h~/dt2.
 * kappa = (5/3) t f(y), y = (2/3) t^{-3/2}, f(y) = eta - (2/3) I_{3/2}/y.
 * Derivatives by the chain rule through y(t) and eta(y):
 *   dy/dt = -(3/2) y/t,  deta/dy = 1/I'_{1/2} = 2/I_{-1/2},  df/dy = (2/3) I_{3/2}/y^2.
 */
int oracle_kappa_h(long n, const double *tin, double *out)
{
    gl_init();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        double t = tin[i];
        double y = (2.0 / 3.0) * pow(t, -1.5);
        double eta = eta_of_y(y);
        double m[6];
        fd_moments(eta, m, 6);
        double Im = m[0], Ih = m[1], I3 = m[2], Ip = m[3], Ipp = m[4], Ippp = m[5];

        /* kappa and its t-derivatives (footnote a of Table I). */
        double fy = eta - (2.0 / 3.0) * I3 / y;
        double kap = (5.0 / 3.0) * t * fy;
        double dy = -1.5 * y / t;
        double dfy = (2.0 / 3.0) * I3 / (y * y);
        double dkap = (5.0 / 3.0) * (fy + t * dfy * dy);
        /* d2kappa/dt2: differentiate (5/3)[eta - (5/3) I_{3/2}/y] (the simplified dkap). */
        double deta = (2.0 / Im) * dy;               /* deta/dt */
        double dI3 = 1.5 * Ih * deta;                /* I'_{3/2} = (3/2) I_{1/2} */
        double d2kap = (5.0 / 3.0) * (deta - (5.0 / 3.0) * (dI3 / y - I3 * dy / (y * y)));

        /* h~(eta) = 6 N/D with N = I_{1/2} I'_{-1/2}, D = I_{-1/2}^2. */
        double a = Ih, a1 = 0.5 * Im, a2 = 0.5 * Ip;
        double b = Ip, b1 = Ipp, b2 = Ippp;
        double Nn = a * b, N1 = a1 * b + a * b1, N2 = a2 * b + 2.0 * a1 * b1 + a * b2;
        double D = Im * Im, D1 = 2.0 * Im * Ip, D2 = 2.0 * Ip * Ip + 2.0 * Im * Ipp;
        double H = 6.0 * Nn / D;
        double He = 6.0 * (N1 / D - Nn * D1 / (D * D));
        double Hee = 6.0 * (N2 / D - 2.0 * N1 * D1 / (D * D) - Nn * D2 / (D * D) + 2.0 * Nn * D1 * D1 / (D * D * D));
        /* eta(t): deta/dt = -2 t^{-5/2}/I_{-1/2}; second derivative by the quotient rule. */
        double et = -2.0 * pow(t, -2.5) / Im;
        double ett = 5.0 * pow(t, -3.5) / Im + 2.0 * pow(t, -2.5) * Ip * et / (Im * Im);
        double ht = He * et;
        double htt = Hee * et * et + He * ett;

        double *o = out + 7 * i;
        o[0] = eta; o[1] = kap; o[2] = dkap; o[3] = d2kap;
        o[4] = H; o[5] = ht; o[6] = htt;
    }
    return 0;
}
