// C ABI of libofdft (include/ofdft.h): context, evaluation pipeline, CG
// minimiser, forces, pressure and MD driver.  Host code only orders kernels
// on the context's stream and reads back a handful of reduced scalars.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "pointwise.cuh"

using namespace ofdft;

namespace {

const double kPi = 3.14159265358979323846;
const double kKbHa = 3.166811563e-6;        // hartree / kelvin
const double kFsAu = 41.341373335;          // atomic time units per fs
const double kMassH = 1.00794 * 1822.888486209;

std::string g_setup_error;

struct Scal {
    double v[24];
};

}  // namespace

struct ofdft_ctx {
    int dev = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    GridInfo g{};
    int nat = 0;
    std::vector<double> R, Z, masses;
    double T = 0.0;             // hartree
    int functional = 0;
    FuncParams fp{};
    int xc = 1;
    int precision = 0;
    double Ne = 0.0;
    FftAxis ax[2][3];           // [precision 0 = double, 1 = float][x, y, z]
    void *tw[2][3] = {{nullptr}};
    // fields (sized for double)
    void *phi = nullptr, *phit = nullptr, *dhat = nullptr, *gv = nullptr, *gprev = nullptr,
         *d = nullptr, *v = nullptr, *vt = nullptr, *vpart = nullptr, *phiprev = nullptr;
    void *spec[4] = {nullptr, nullptr, nullptr, nullptr};
    void *vext[2] = {nullptr, nullptr};
    void *tab[2] = {nullptr, nullptr};
    double *part = nullptr;
    size_t part_len = 0;
    double *scal = nullptr;
    double *scal_h = nullptr;
    // ions
    double *Rd = nullptr, *Zd = nullptr, *Fd = nullptr, *Vd = nullptr, *Md = nullptr, *nh = nullptr;
    double2 *px = nullptr, *py = nullptr, *pz = nullptr;
    double *fpart = nullptr;
    size_t fpart_len = 0;
    // Ewald
    double *Gv = nullptr, *wG = nullptr, *eion = nullptr, *ewF = nullptr, *ewpart = nullptr, *Ld = nullptr;
    double2 *Se = nullptr;
    int nGe = 0;
    double ew_alpha = 0.0, ew_rcut = 0.0;
    int3 ew_nimg{0, 0, 0};
    double E_ion = 0.0;
    // state
    ofdft_energy last{};
    bool last_valid = false;
    bool md_ready = false;
    double md_kT = 0.0, md_Q = 1.0, md_dt = 0.0;
    int md_thermo = 0;
    long long launches = 0;
    std::string err;
    // kernel timer (diagnostics)
    int timer_id = 0;
    std::vector<cudaEvent_t> tev;
    size_t tev_used = 0;
};

namespace {

#define CK(call)                                                                 \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e_), #call); \
    } while (0)

ofdft_status fail(ofdft_ctx *c, ofdft_status s, const char *msg, const char *where = nullptr)
{
    std::string m = msg ? msg : "error";
    if (where) m += std::string(" at ") + where;
    if (c) c->err = m;
    else g_setup_error = m;
    return s;
}

bool smooth_even(int n)
{
    if (n < 8 || n > 512 || (n & 1)) return false;
    int m = n;
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

FftAxis make_axis(int n)
{
    FftAxis a{};
    a.n = n;
    int m = n, ns = 1, k = 0;
    for (int r : {8, 4, 2, 3, 5}) {
        while (m % r == 0) {
            a.rad[k] = r;
            a.ns[k] = ns;
            ns *= r;
            m /= r;
            ++k;
        }
    }
    a.nst = k;
    return a;
}

template <typename T> ofdft_status upload_twiddles(ofdft_ctx *c, int prec, int axis, int n)
{
    std::vector<cplx<T>> w(n);
    for (int m = 0; m < n; ++m) {
        long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)n;
        w[m].x = (T)cosl(ang);
        w[m].y = (T)sinl(ang);
    }
    CK(cudaMalloc(&c->tw[prec][axis], n * sizeof(cplx<T>)));
    CK(cudaMemcpy(c->tw[prec][axis], w.data(), n * sizeof(cplx<T>), cudaMemcpyHostToDevice));
    c->ax[prec][axis] = make_axis(n);
    c->ax[prec][axis].tw = c->tw[prec][axis];
    return OFDFT_OK;
}

ofdft_status ensure_part(ofdft_ctx *c, size_t n)
{
    if (n <= c->part_len) return OFDFT_OK;
    if (c->part) cudaFree(c->part);
    c->part = nullptr;
    CK(cudaMalloc(&c->part, n * sizeof(double)));
    c->part_len = n;
    return OFDFT_OK;
}

ofdft_status sync_read(ofdft_ctx *c, int n)
{
    CK(cudaMemcpyAsync(c->scal_h, c->scal, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaGetLastError());
    return OFDFT_OK;
}

// ------------------------------------------------------------ evaluation
// Scalar block after an evaluation: [0] E_H [1] E_loc [2] P_loc,
// [3..8] GGA pointwise partials, [9..17] final-stage partials.
enum TimerId { TM_ZGGA = 1, TM_XGRAD = 2, TM_XDIV = 3, TM_Y = 4, TM_ZFWD = 5, TM_ZFINAL = 6, TM_XHL = 7 };

// Event pair around a launch of the selected kernel class.
struct TimerScope {
    ofdft_ctx *c;
    bool on;
    TimerScope(ofdft_ctx *c_, int id) : c(c_), on(c_->timer_id == id)
    {
        if (!on) return;
        if (c->tev_used + 2 > c->tev.size()) {
            for (int i = 0; i < 256; ++i) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                c->tev.push_back(e);
            }
        }
        cudaEventRecord(c->tev[c->tev_used], c->st);
    }
    ~TimerScope()
    {
        if (!on) return;
        cudaEventRecord(c->tev[c->tev_used + 1], c->st);
        c->tev_used += 2;
    }
};

struct EvalScalars {
    double EH, Eloc, Ploc, FS, TS, FXC, PS, WG, PXC, PHI2V, PHI2, DTH;
};

template <typename T>
ofdft_status evaluate(ofdft_ctx *c, T *ph, const T *phi0, const T *dh, double cth, double sth,
                      T *vout, bool keep_nG, EvalScalars &es)
{
    const int pi = sizeof(T) == 8 ? 0 : 1;
    const GridInfo &g = c->g;
    const FftAxis &ax = c->ax[pi][0], &ay = c->ax[pi][1], &az = c->ax[pi][2];
    cudaStream_t st = c->st;
    typedef cplx<T> C;
    C *s0 = (C *)c->spec[0], *s1 = (C *)c->spec[1], *s2 = (C *)c->spec[2], *s3 = (C *)c->spec[3];
    const C *vext = (const C *)c->vext[pi];
    const T *tab = (const T *)c->tab[pi];
    const long long NH = s1 - s0;          // field stride of the spectrum block, in elements
    const bool fttf = c->fp.kind == 0;
    // part regions: A (x pass, 3 q), B (zgga, 6 q), C (zfinal, 9 q)
    int ntk = (g.K + 7) / 8;
    int nbx = g.ny * ntk;
    long long npairs = (long long)g.nx * g.ny / 2;
    size_t need = (size_t)3 * nbx + (size_t)15 * (size_t)npairs + 64;
    if (ensure_part(c, need) != OFDFT_OK) return OFDFT_ENOMEM;
    double *pA = c->part, *pB = pA + 3 * nbx, *pC = pB + 6 * npairs;
    {
        TimerScope ts(c, TM_ZFWD);
        if (phi0) launch_zfwd<T>(g, az, 2, nullptr, phi0, dh, (T)cth, (T)sth, ph, s0, st);
        else launch_zfwd<T>(g, az, 1, nullptr, ph, nullptr, T(0), T(0), nullptr, s0, st);
    }
    {
        TimerScope ts(c, TM_Y);
        launch_ypass<T>(g, ay, false, s0, 1, NH, st);
    }
    int nbz;
    if (fttf) {
        {
            TimerScope ts(c, TM_XHL);
            launch_xhl<T>(g, ax, s0, vext, keep_nG ? s1 : nullptr, 1, pA, st);
        }
        {
            TimerScope ts(c, TM_Y);
            launch_ypass<T>(g, ay, true, s0, 1, NH, st);
        }
        TimerScope ts(c, TM_ZFINAL);
        nbz = launch_zfinal<T>(g, az, true, s0, nullptr, ph, phi0, dh, (T)cth, (T)sth, (T)c->T, c->fp,
                               tab, c->xc, vout, pC, st);
        c->launches += 5;
    } else {
        {
            TimerScope ts(c, TM_XGRAD);
            launch_xgrad<T>(g, ax, s0, vext, s1, s2, s3, pA, st);
        }
        {
            TimerScope ts(c, TM_Y);
            launch_ypass<T>(g, ay, true, s1, 3, NH, st);
        }
        {
            TimerScope ts(c, TM_ZGGA);
            launch_zgga<T>(g, az, s1, s2, s3, ph, (T)c->T, c->fp, tab, c->xc, (T *)c->vpart, pB, st);
        }
        {
            TimerScope ts(c, TM_Y);
            launch_ypass<T>(g, ay, false, s1, 3, NH, st);
        }
        {
            TimerScope ts(c, TM_XDIV);
            launch_xdiv<T>(g, ax, s0, vext, s1, s2, s3, st);
        }
        {
            TimerScope ts(c, TM_Y);
            launch_ypass<T>(g, ay, true, s1, 1, NH, st);
        }
        TimerScope ts(c, TM_ZFINAL);
        nbz = launch_zfinal<T>(g, az, false, s1, (const T *)c->vpart, ph, phi0, dh, (T)cth, (T)sth,
                               (T)c->T, c->fp, tab, c->xc, vout, pC, st);
        c->launches += 9;
    }
    launch_reduce(pA, nbx, 3, c->scal, st);
    if (!fttf) launch_reduce(pB, nbz, 6, c->scal + 3, st);
    launch_reduce(pC, nbz, 9, c->scal + 9, st);
    c->launches += fttf ? 2 : 3;
    if (sync_read(c, 18) != OFDFT_OK) return OFDFT_EDEVICE;
    const double *h = c->scal_h;
    es.EH = h[0];
    es.Eloc = h[1];
    es.Ploc = h[2];
    const double *f = fttf ? h + 9 : h + 3;
    es.FS = f[0];
    es.TS = f[1];
    es.FXC = f[2];
    es.PS = f[3];
    es.WG = fttf ? 0.0 : f[4];
    es.PXC = f[5];
    es.PHI2V = h[15];
    es.PHI2 = h[16];
    es.DTH = h[17];
    double chk = es.EH + es.Eloc + es.FS + es.FXC + es.PHI2V + es.DTH;
    if (!isfinite(chk)) return fail(c, OFDFT_ENUMERIC, "non-finite energy or potential");
    return OFDFT_OK;
}

void fill_energy(const ofdft_ctx *c, const EvalScalars &es, ofdft_energy &E)
{
    const double dV = c->g.dV, om = c->g.omega;
    memset(&E, 0, sizeof(E));
    E.F_s = dV * es.FS;
    E.minus_TS = -dV * es.TS;
    E.E_H = es.EH;
    E.E_loc = es.Eloc;
    E.F_xc = dV * es.FXC;
    E.E_ion = c->E_ion;
    E.F_tot = E.F_s + E.E_H + E.E_loc + E.F_xc + E.E_ion;
    E.E_int = E.F_tot + dV * es.TS;
    E.mu = es.PHI2V / es.PHI2;
    double zs = 0.0;
    for (int i = 0; i < c->nat; ++i) zs += kPi * c->Z[i] * c->g.rc * c->g.rc;
    E.E_alphaZ = c->Ne * zs / om;
    E.P_s = (dV * es.PS + (4.0 / 3.0) * dV * es.WG) / om;
    E.P_xc = dV * es.PXC / om;
    E.P_H = es.EH / (3.0 * om);
    E.P_loc = es.Ploc;
    E.P_ion = c->E_ion / (3.0 * om);
    E.P = E.P_s + E.P_xc + E.P_H + E.P_loc + E.P_ion;
}

// ---------------------------------------------------------- ions & Ewald
ofdft_status setup_ewald(ofdft_ctx *c)
{
    const GridInfo &g = c->g;
    double L[3] = {g.Lx, g.Ly, g.Lz};
    double om = g.omega;
    c->ew_alpha = 1.2 * sqrt(kPi) * pow((double)c->nat / (om * om), 1.0 / 6.0);
    c->ew_rcut = 6.3 / c->ew_alpha;
    c->ew_nimg = make_int3((int)ceil(c->ew_rcut / L[0] + 0.5), (int)ceil(c->ew_rcut / L[1] + 0.5),
                           (int)ceil(c->ew_rcut / L[2] + 0.5));
    double gcut = 2.0 * c->ew_alpha * 6.3;
    int km[3];
    for (int a = 0; a < 3; ++a) km[a] = (int)ceil(gcut * L[a] / (2.0 * kPi));
    std::vector<double> Gv, wG;
    for (int i = -km[0]; i <= km[0]; ++i)
        for (int j = -km[1]; j <= km[1]; ++j)
            for (int k = -km[2]; k <= km[2]; ++k) {
                double gx = 2 * kPi * i / L[0], gy = 2 * kPi * j / L[1], gz = 2 * kPi * k / L[2];
                double g2 = gx * gx + gy * gy + gz * gz;
                if (g2 == 0.0 || g2 >= gcut * gcut) continue;
                Gv.push_back(gx);
                Gv.push_back(gy);
                Gv.push_back(gz);
                wG.push_back(2.0 * kPi / om * exp(-g2 / (4.0 * c->ew_alpha * c->ew_alpha)) / g2);
            }
    c->nGe = (int)wG.size();
    int nb = (c->nGe + 255) / 256;
    CK(cudaMalloc(&c->Gv, std::max<size_t>(1, Gv.size()) * sizeof(double)));
    CK(cudaMalloc(&c->wG, std::max<size_t>(1, wG.size()) * sizeof(double)));
    CK(cudaMalloc(&c->Se, std::max(1, c->nGe) * sizeof(double2)));
    CK(cudaMalloc(&c->ewpart, std::max(1, nb) * sizeof(double)));
    CK(cudaMalloc(&c->eion, c->nat * sizeof(double)));
    CK(cudaMalloc(&c->ewF, 3 * c->nat * sizeof(double)));
    CK(cudaMalloc(&c->Ld, 3 * sizeof(double)));
    if (!Gv.empty()) {
        CK(cudaMemcpy(c->Gv, Gv.data(), Gv.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->wG, wG.data(), wG.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(c->Ld, L, 3 * sizeof(double), cudaMemcpyHostToDevice));
    return OFDFT_OK;
}

// Recompute v_ext(G) (both precisions) and the Ewald energy and forces from Rd.
ofdft_status update_ions(ofdft_ctx *c)
{
    const GridInfo &g = c->g;
    cudaStream_t st = c->st;
    launch_phases(g, c->nat, c->Rd, c->px, c->py, c->pz, st);
    launch_vext<double>(g, c->nat, c->Zd, c->px, c->py, c->pz, (double2 *)c->vext[0], st);
    if (c->precision == OFDFT_MIXED)
        launch_vext<float>(g, c->nat, c->Zd, c->px, c->py, c->pz, (float2 *)c->vext[1], st);
    double L[3] = {g.Lx, g.Ly, g.Lz};
    launch_ewald_real(c->nat, c->Rd, c->Zd, L, c->ew_alpha, c->ew_rcut, c->ew_nimg, c->eion, c->ewF, st);
    int nb = launch_ewald_recip(c->nat, c->Rd, c->Zd, c->nGe, c->Gv, c->wG, c->Se, c->ewpart, c->ewF, st);
    c->launches += 5 + (c->precision == OFDFT_MIXED);
    std::vector<double> e(c->nat + nb);
    CK(cudaMemcpyAsync(e.data(), c->eion, c->nat * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(e.data() + c->nat, c->ewpart, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    double E = 0.0;
    for (double x : e) E += x;
    double z2 = 0.0, zs = 0.0;
    for (int i = 0; i < c->nat; ++i) {
        z2 += c->Z[i] * c->Z[i];
        zs += c->Z[i];
    }
    E -= c->ew_alpha / sqrt(kPi) * z2;
    E -= kPi * zs * zs / (2.0 * g.omega * c->ew_alpha * c->ew_alpha);
    c->E_ion = E;
    c->last_valid = false;
    return OFDFT_OK;
}

// ------------------------------------------------------------------- CG
template <typename T> ofdft_status normalize_phi(ofdft_ctx *c, T *x)
{
    if (ensure_part(c, 4096) != OFDFT_OK) return OFDFT_ENOMEM;
    int nb = launch_sumsq<T>(c->g.N, x, c->part, c->st);
    launch_reduce(c->part, nb, 1, c->scal, c->st);
    c->launches += 2;
    if (sync_read(c, 1) != OFDFT_OK) return OFDFT_EDEVICE;
    double ss = c->scal_h[0] * c->g.dV;
    if (!(ss > 0.0) || !isfinite(ss)) return fail(c, OFDFT_ENUMERIC, "phi has zero or non-finite norm");
    launch_scale<T>(c->g.N, x, sqrt(c->Ne / ss), c->st);
    c->launches++;
    return OFDFT_OK;
}

struct LsResult {
    bool ok;
    double theta;
    int nevals;
    EvalScalars es;
};

template <typename T>
ofdft_status line_search(ofdft_ctx *c, double D0, double theta1, LsResult &r)
{
    const double ls_tol = 0.1;
    const int max_ls = 20;
    double lo = 0.0, Dlo = D0, hi = -1.0, Dhi = 0.0, pa = 0.0, Da = D0, th = theta1;
    r.ok = false;
    r.nevals = 0;
    for (int k = 0; k < max_ls; ++k) {
        EvalScalars es;
        ofdft_status s = evaluate<T>(c, (T *)c->phit, (const T *)c->phi, (const T *)c->dhat, cos(th),
                                     sin(th), (T *)c->vt, false, es);
        r.nevals++;
        if (s != OFDFT_OK) return s;
        double D = c->g.dV * es.DTH;
        if (fabs(D) <= ls_tol * fabs(D0)) {
            r.ok = true;
            r.theta = th;
            r.es = es;
            return OFDFT_OK;
        }
        if (D < 0.0) {
            lo = th;
            Dlo = D;
        } else {
            hi = th;
            Dhi = D;
        }
        double nxt;
        if (hi < 0.0) {
            nxt = 4.0 * th;
            if (D > Da) {
                double sec = th - D * (th - pa) / (D - Da);
                nxt = std::min(sec, 4.0 * th);
            }
            nxt = std::max(nxt, 1.1 * th);
            pa = th;
            Da = D;
        } else {
            nxt = lo - Dlo * (hi - lo) / (Dhi - Dlo);
            double w = hi - lo;
            nxt = std::min(std::max(nxt, lo + 0.01 * w), hi - 0.01 * w);
        }
        th = std::min(nxt, 1.5);
    }
    if (lo > 0.0) {
        EvalScalars es;
        ofdft_status s = evaluate<T>(c, (T *)c->phit, (const T *)c->phi, (const T *)c->dhat, cos(lo),
                                     sin(lo), (T *)c->vt, false, es);
        r.nevals++;
        if (s != OFDFT_OK) return s;
        r.ok = true;
        r.theta = lo;
        r.es = es;
    }
    return OFDFT_OK;
}

template <typename T>
ofdft_status minimize_T(ofdft_ctx *c, double gtol, int maxit, ofdft_stats &stats, EvalScalars &es_out)
{
    const long long N = c->g.N;
    const double dV = c->g.dV;
    cudaStream_t st = c->st;
    stats.iterations = 0;
    stats.evaluations = 0;
    stats.gnorm = 0.0;
    stats.status = OFDFT_OK;
    ofdft_status s = normalize_phi<T>(c, (T *)c->phi);
    if (s != OFDFT_OK) return s;
    EvalScalars es;
    s = evaluate<T>(c, (T *)c->phi, nullptr, nullptr, 1.0, 0.0, (T *)c->v, false, es);
    stats.evaluations = 1;
    if (s != OFDFT_OK) return s;
    if (ensure_part(c, 8 * 1216) != OFDFT_OK) return OFDFT_ENOMEM;
    double mu = es.PHI2V / es.PHI2;
    int nb = launch_cg_grad<T>(N, (const T *)c->phi, (const T *)c->v, mu, (T *)c->gv, nullptr, c->part, st);
    launch_reduce(c->part, nb, 2, c->scal, st);
    c->launches += 2;
    if (sync_read(c, 2) != OFDFT_OK) return OFDFT_EDEVICE;
    double gg = c->scal_h[0], ggprev = 0.0;
    double gnorm = sqrt(dV * gg);
    bool have_prev = false;
    double theta_prev = 0.05;
    int it = 0;
    ofdft_status status = OFDFT_ENOCONV;
    while (it < maxit) {
        if (gnorm < gtol) {
            status = OFDFT_OK;
            break;
        }
        double beta = 0.0;
        if (have_prev) beta = std::max(0.0, (gg - c->scal_h[1]) / ggprev);
        nb = launch_cg_dir<T>(N, (const T *)c->gv, (T *)c->d, have_prev ? beta : 0.0,
                              (const T *)c->phi, c->part, st);
        launch_reduce(c->part, nb, 5, c->scal + 4, st);
        c->launches += 2;
        if (sync_read(c, 9) != OFDFT_OK) return OFDFT_EDEVICE;
        double sphd = c->scal_h[4], sdd = c->scal_h[5], sdg = c->scal_h[6], spp = c->scal_h[7],
               spg = c->scal_h[8];
        double c1 = sphd / spp;
        double dg = sdg - c1 * spg;
        double dd = sdd - 2.0 * c1 * sphd + c1 * c1 * spp;
        int restart = dg >= 0.0;
        double c2 = restart ? sqrt(spp / gg) : sqrt(spp / dd);
        nb = launch_cg_dhat<T>(N, (const T *)c->gv, (T *)c->d, (const T *)c->phi, (const T *)c->v, c1, c2,
                               restart, (T *)c->dhat, c->part, st);
        launch_reduce(c->part, nb, 1, c->scal, st);
        c->launches += 2;
        if (sync_read(c, 1) != OFDFT_OK) return OFDFT_EDEVICE;
        double D0 = dV * c->scal_h[0];
        LsResult ls;
        s = line_search<T>(c, D0, theta_prev, ls);
        stats.evaluations += ls.nevals;
        if (s != OFDFT_OK) return s;
        if (!ls.ok) {
            if (!have_prev) {
                status = OFDFT_ENOCONV;
                break;
            }
            have_prev = false;   // restart along steepest descent
            continue;
        }
        theta_prev = ls.theta;
        std::swap(c->phi, c->phit);
        std::swap(c->v, c->vt);
        es = ls.es;
        std::swap(c->gv, c->gprev);
        mu = es.PHI2V / es.PHI2;
        nb = launch_cg_grad<T>(N, (const T *)c->phi, (const T *)c->v, mu, (T *)c->gv, (const T *)c->gprev,
                               c->part, st);
        launch_reduce(c->part, nb, 2, c->scal, st);
        c->launches += 2;
        if (sync_read(c, 2) != OFDFT_OK) return OFDFT_EDEVICE;
        ggprev = gg;
        gg = c->scal_h[0];
        gnorm = sqrt(dV * gg);
        have_prev = true;
        ++it;
    }
    if (gnorm < gtol) status = OFDFT_OK;
    stats.iterations = it;
    stats.gnorm = gnorm;
    stats.status = status;
    es_out = es;
    return OFDFT_OK;
}

// Final FP64 evaluation at the current phi; for MIXED contexts phi is FP32
// and is widened into the phit buffer first.
ofdft_status eval_fp64_at_phi(ofdft_ctx *c, bool keep_nG, EvalScalars &es, double **phi64)
{
    double *ph = (double *)c->phi;
    if (c->precision == OFDFT_MIXED) {
        launch_convert<float, double>(c->g.N, (const float *)c->phi, (double *)c->phit, c->st);
        c->launches++;
        ph = (double *)c->phit;
    }
    if (phi64) *phi64 = ph;
    return evaluate<double>(c, ph, nullptr, nullptr, 1.0, 0.0, (double *)c->vt, keep_nG, es);
}

ofdft_status forces_now(ofdft_ctx *c, EvalScalars &es)
{
    ofdft_status s = eval_fp64_at_phi(c, true, es, nullptr);
    if (s != OFDFT_OK) return s;
    const GridInfo &g = c->g;
    const double2 *nG = (const double2 *)(c->fp.kind == 0 ? c->spec[1] : c->spec[0]);
    size_t need = (size_t)c->nat * 608 * 3 + 16;
    if (need > c->fpart_len) {
        if (c->fpart) cudaFree(c->fpart);
        c->fpart = nullptr;
        CK(cudaMalloc(&c->fpart, need * sizeof(double)));
        c->fpart_len = need;
    }
    int nchunk = launch_lpp_forces<double>(g, c->nat, c->Zd, c->px, c->py, c->pz, nG, c->fpart, c->st);
    launch_force_reduce(c->nat, nchunk, c->fpart, c->Fd, 0, c->st);
    c->launches += 2;
    // add Ewald forces
    std::vector<double> F(3 * c->nat), Fe(3 * c->nat);
    CK(cudaMemcpyAsync(F.data(), c->Fd, F.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(Fe.data(), c->ewF, Fe.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (size_t i = 0; i < F.size(); ++i) F[i] += Fe[i];
    CK(cudaMemcpyAsync(c->Fd, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    return OFDFT_OK;
}

ofdft_status run_minimize(ofdft_ctx *c, double gtol, int maxit, ofdft_stats &stats, EvalScalars &es)
{
    ofdft_status s;
    if (c->precision == OFDFT_MIXED) {
        double gt = std::max(gtol, 1e-5);
        s = minimize_T<float>(c, gt, maxit, stats, es);
        if (s != OFDFT_OK) return s;
        EvalScalars e64;
        s = eval_fp64_at_phi(c, false, e64, nullptr);
        stats.evaluations++;
        if (s != OFDFT_OK) return s;
        es = e64;
    } else {
        s = minimize_T<double>(c, gtol, maxit, stats, es);
        if (s != OFDFT_OK) return s;
    }
    fill_energy(c, es, c->last);
    c->last_valid = true;
    return stats.status == OFDFT_OK ? OFDFT_OK : (ofdft_status)stats.status;
}

void free_ctx(ofdft_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->st) cudaStreamSynchronize(c->st);
    void *ptrs[] = {c->phi, c->phit, c->dhat, c->gv, c->gprev, c->d, c->v, c->vt, c->vpart, c->phiprev,
                    c->spec[0], c->vext[0], c->vext[1],
                    c->tab[0], c->tab[1], c->part, c->scal, c->Rd, c->Zd, c->Fd, c->Vd, c->Md,
                    c->nh, c->px, c->py, c->pz, c->fpart, c->Gv, c->wG, c->eion, c->ewF, c->ewpart,
                    c->Ld, c->Se, c->tw[0][0], c->tw[0][1], c->tw[0][2], c->tw[1][0], c->tw[1][1],
                    c->tw[1][2]};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->scal_h) cudaFreeHost(c->scal_h);
    for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c;
}

ofdft_status alloc_ctx(ofdft_ctx *c)
{
    const GridInfo &g = c->g;
    size_t rb = (size_t)g.N * sizeof(double), cb = (size_t)g.NH * sizeof(double2);
    void **fields[] = {&c->phi, &c->phit, &c->dhat, &c->gv, &c->gprev, &c->d, &c->v, &c->vt, &c->vpart,
                       &c->phiprev};
    for (void **f : fields) CK(cudaMalloc(f, rb));
    // the four half spectra are one allocation: the y pass walks fields 1..3
    // with a fixed stride
    CK(cudaMalloc(&c->spec[0], 4 * cb));
    for (int i = 1; i < 4; ++i) c->spec[i] = (char *)c->spec[0] + i * cb;
    CK(cudaMalloc(&c->vext[0], cb));
    if (c->precision == OFDFT_MIXED) CK(cudaMalloc(&c->vext[1], (size_t)g.NH * sizeof(float2)));
    CK(cudaMalloc(&c->scal, 64 * sizeof(double)));
    CK(cudaMallocHost(&c->scal_h, 64 * sizeof(double)));
    const int nat = c->nat;
    CK(cudaMalloc(&c->Rd, 3 * nat * sizeof(double)));
    CK(cudaMalloc(&c->Zd, nat * sizeof(double)));
    CK(cudaMalloc(&c->Fd, 3 * nat * sizeof(double)));
    CK(cudaMalloc(&c->Vd, 3 * nat * sizeof(double)));
    CK(cudaMalloc(&c->Md, nat * sizeof(double)));
    CK(cudaMalloc(&c->nh, 4 * sizeof(double)));
    CK(cudaMalloc(&c->px, (size_t)nat * g.nx * sizeof(double2)));
    CK(cudaMalloc(&c->py, (size_t)nat * g.ny * sizeof(double2)));
    CK(cudaMalloc(&c->pz, (size_t)nat * g.K * sizeof(double2)));
    // temperature tables
    const std::vector<double> &tab = tfunc_table_host();
    CK(cudaMalloc(&c->tab[0], tab.size() * sizeof(double)));
    CK(cudaMemcpy(c->tab[0], tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<float> tabf(tab.begin(), tab.end());
    CK(cudaMalloc(&c->tab[1], tabf.size() * sizeof(float)));
    CK(cudaMemcpy(c->tab[1], tabf.data(), tabf.size() * sizeof(float), cudaMemcpyHostToDevice));
    int n3[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        if (upload_twiddles<double>(c, 0, a, n3[a]) != OFDFT_OK) return OFDFT_EDEVICE;
        if (upload_twiddles<float>(c, 1, a, n3[a]) != OFDFT_OK) return OFDFT_EDEVICE;
    }
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
    if (field_smem_max(g, sizeof(double2)) > (size_t)optin)
        return fail(c, OFDFT_EINVAL, "grid too large for the shared-memory tiles");
    set_field_smem_limits<double>((size_t)optin);
    set_field_smem_limits<float>((size_t)optin);
    CK(cudaGetLastError());
    return OFDFT_OK;
}

}  // namespace

FuncParams ofdft::functional_params(int f)
{
    FuncParams p{};
    switch (f) {
    case OFDFT_FTTF: p.kind = 0; break;
    case OFDFT_SGA: p.kind = 1; p.p0 = 5.0 / 27.0; break;
    case OFDFT_VWTF: p.kind = 1; p.p0 = 5.0 / 3.0; break;
    case OFDFT_VT84F: p.kind = 2; break;
    case OFDFT_KST2: p.kind = 3; p.p0 = 2.03087; p.p1 = 0.29424; break;
    case OFDFT_TW: p.kind = 3; p.p0 = 0.2319; p.p1 = 0.2748; break;
    case OFDFT_APBEF: p.kind = 3; p.p0 = 0.23889; p.p1 = 0.23889 / 0.804; break;
    default: p.kind = -1;
    }
    return p;
}

// ====================================================================== ABI
extern "C" {

void ofdft_default_params(ofdft_params *p)
{
    if (!p) return;
    p->xc = 1;
    p->rc = 0.25;
    p->precision = OFDFT_FP64;
    p->device = 0;
    p->stream = nullptr;
}

ofdft_status ofdft_setup(const double cell[9], const int grid[3], int nat, const double *ions,
                         const double *Z, double T_kelvin, int functional, const ofdft_params *params,
                         ofdft_ctx **out)
{
    if (!out) return fail(nullptr, OFDFT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cell || !grid || !ions || !Z || nat <= 0) return fail(nullptr, OFDFT_EINVAL, "NULL input or nat <= 0");
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (i != j && cell[3 * i + j] != 0.0)
                return fail(nullptr, OFDFT_EINVAL, "cell is not orthorhombic");
    if (!(cell[0] > 0 && cell[4] > 0 && cell[8] > 0)) return fail(nullptr, OFDFT_EINVAL, "non-positive cell edge");
    for (int a = 0; a < 3; ++a)
        if (!smooth_even(grid[a]))
            return fail(nullptr, OFDFT_EINVAL, "grid edges must be even, {2,3,5}-smooth, in [8, 512]");
    if (!(T_kelvin > 0.0) || !isfinite(T_kelvin)) return fail(nullptr, OFDFT_EINVAL, "temperature must be > 0");
    FuncParams fp = functional_params(functional);
    if (fp.kind < 0) return fail(nullptr, OFDFT_EINVAL, "unknown functional");
    ofdft_params p;
    ofdft_default_params(&p);
    if (params) p = *params;
    if (!(p.rc > 0.0)) return fail(nullptr, OFDFT_EINVAL, "rc must be > 0");
    if (p.precision != OFDFT_FP64 && p.precision != OFDFT_MIXED) return fail(nullptr, OFDFT_EINVAL, "bad precision");
    for (int i = 0; i < nat; ++i) {
        if (!(Z[i] > 0.0)) return fail(nullptr, OFDFT_EINVAL, "Z must be > 0");
        for (int a = 0; a < 3; ++a)
            if (!isfinite(ions[3 * i + a])) return fail(nullptr, OFDFT_EINVAL, "non-finite ion position");
    }
    ofdft_ctx *c = new (std::nothrow) ofdft_ctx();
    if (!c) return fail(nullptr, OFDFT_ENOMEM, "host allocation failed");
    c->dev = p.device;
    if (cudaSetDevice(c->dev) != cudaSuccess) {
        delete c;
        return fail(nullptr, OFDFT_EDEVICE, "cudaSetDevice failed");
    }
    if (p.stream) {
        c->st = (cudaStream_t)p.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(nullptr, OFDFT_EDEVICE, "stream creation failed");
        }
        c->own_stream = true;
    }
    GridInfo &g = c->g;
    g.nx = grid[0];
    g.ny = grid[1];
    g.nz = grid[2];
    g.K = g.nz / 2 + 1;
    g.N = (long long)g.nx * g.ny * g.nz;
    g.NH = (long long)g.nx * g.ny * g.K;
    g.Lx = cell[0];
    g.Ly = cell[4];
    g.Lz = cell[8];
    g.omega = g.Lx * g.Ly * g.Lz;
    g.dV = g.omega / (double)g.N;
    g.rc = p.rc;
    c->nat = nat;
    c->R.assign(ions, ions + 3 * nat);
    c->Z.assign(Z, Z + nat);
    c->masses.assign(nat, kMassH);
    c->T = T_kelvin * kKbHa;
    c->functional = functional;
    c->fp = fp;
    c->xc = p.xc;
    c->precision = p.precision;
    c->Ne = 0.0;
    for (int i = 0; i < nat; ++i) c->Ne += Z[i];
    ofdft_status s = alloc_ctx(c);
    if (s == OFDFT_OK) s = setup_ewald(c);
    if (s != OFDFT_OK) {
        g_setup_error = c->err;
        free_ctx(c);
        return s == OFDFT_EDEVICE ? OFDFT_ENOMEM : s;
    }
    cudaMemcpy(c->Rd, c->R.data(), 3 * nat * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->Zd, c->Z.data(), nat * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->Md, c->masses.data(), nat * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemset(c->Vd, 0, 3 * nat * sizeof(double));
    cudaMemset(c->nh, 0, 4 * sizeof(double));
    s = update_ions(c);
    if (s == OFDFT_OK) s = ofdft_set_phi(c, nullptr);
    if (s != OFDFT_OK) {
        g_setup_error = c->err;
        free_ctx(c);
        return s;
    }
    *out = c;
    return OFDFT_OK;
}

ofdft_status ofdft_set_positions(ofdft_ctx *c, const double *ions)
{
    if (!c || !ions) return fail(c, OFDFT_EINVAL, "NULL argument");
    cudaSetDevice(c->dev);
    for (int i = 0; i < 3 * c->nat; ++i)
        if (!isfinite(ions[i])) return fail(c, OFDFT_EINVAL, "non-finite ion position");
    c->R.assign(ions, ions + 3 * c->nat);
    CK(cudaMemcpyAsync(c->Rd, c->R.data(), 3 * c->nat * sizeof(double), cudaMemcpyHostToDevice, c->st));
    c->md_ready = false;
    return update_ions(c);
}

ofdft_status ofdft_set_phi(ofdft_ctx *c, const double *phi)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    cudaSetDevice(c->dev);
    const long long N = c->g.N;
    if (phi) {
        if (c->precision == OFDFT_MIXED) {
            CK(cudaMemcpyAsync(c->phit, phi, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
            launch_convert<double, float>(N, (const double *)c->phit, (float *)c->phi, c->st);
            c->launches++;
        } else {
            CK(cudaMemcpyAsync(c->phi, phi, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
        }
    } else {
        double u = sqrt(c->Ne / c->g.omega);
        if (c->precision == OFDFT_MIXED) launch_fill<float>(N, (float *)c->phi, (float)u, c->st);
        else launch_fill<double>(N, (double *)c->phi, u, c->st);
        c->launches++;
    }
    c->last_valid = false;
    c->md_ready = false;
    ofdft_status s = c->precision == OFDFT_MIXED ? normalize_phi<float>(c, (float *)c->phi)
                                                 : normalize_phi<double>(c, (double *)c->phi);
    return s;
}

ofdft_status ofdft_energy_potential(ofdft_ctx *c, const double *phi, ofdft_energy *E, double *v)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    cudaSetDevice(c->dev);
    const long long N = c->g.N;
    double *ph;
    if (phi) {
        CK(cudaMemcpyAsync(c->phit, phi, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
        ph = (double *)c->phit;
    } else if (c->precision == OFDFT_MIXED) {
        launch_convert<float, double>(N, (const float *)c->phi, (double *)c->phit, c->st);
        c->launches++;
        ph = (double *)c->phit;
    } else {
        ph = (double *)c->phi;
    }
    EvalScalars es;
    ofdft_status s = evaluate<double>(c, ph, nullptr, nullptr, 1.0, 0.0, (double *)c->vt, false, es);
    if (s != OFDFT_OK) return s;
    ofdft_energy e;
    fill_energy(c, es, e);
    if (v) {
        CK(cudaMemcpyAsync(v, c->vt, N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    if (E) *E = e;
    return OFDFT_OK;
}

ofdft_status ofdft_minimize(ofdft_ctx *c, double gtol, int maxit, ofdft_energy *E, ofdft_stats *stats)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    if (!(gtol > 0.0) || maxit <= 0) return fail(c, OFDFT_EINVAL, "gtol must be > 0 and maxit > 0");
    cudaSetDevice(c->dev);
    ofdft_stats st{};
    EvalScalars es;
    ofdft_status s = run_minimize(c, gtol, maxit, st, es);
    if (stats) *stats = st;
    if (s != OFDFT_OK && s != OFDFT_ENOCONV) return s;
    if (E) *E = c->last;
    if (s == OFDFT_ENOCONV) return fail(c, OFDFT_ENOCONV, "CG did not reach the tolerance");
    return OFDFT_OK;
}

ofdft_status ofdft_forces(ofdft_ctx *c, double *F, double *pressure)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    cudaSetDevice(c->dev);
    EvalScalars es;
    ofdft_status s = forces_now(c, es);
    if (s != OFDFT_OK) return s;
    ofdft_energy e;
    fill_energy(c, es, e);
    if (F) CK(cudaMemcpy(F, c->Fd, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost));
    if (pressure) *pressure = e.P;
    return OFDFT_OK;
}

ofdft_status ofdft_get_density(ofdft_ctx *c, double *n)
{
    if (!c || !n) return fail(c, OFDFT_EINVAL, "NULL argument");
    cudaSetDevice(c->dev);
    const long long N = c->g.N;
    std::vector<double> tmp;
    if (c->precision == OFDFT_MIXED) {
        launch_convert<float, double>(N, (const float *)c->phi, (double *)c->phit, c->st);
        c->launches++;
        CK(cudaMemcpyAsync(n, c->phit, N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    } else {
        CK(cudaMemcpyAsync(n, c->phi, N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    }
    CK(cudaStreamSynchronize(c->st));
    for (long long i = 0; i < N; ++i) n[i] *= n[i];
    return OFDFT_OK;
}

ofdft_status ofdft_set_masses(ofdft_ctx *c, const double *m)
{
    if (!c || !m) return fail(c, OFDFT_EINVAL, "NULL argument");
    for (int i = 0; i < c->nat; ++i)
        if (!(m[i] > 0.0)) return fail(c, OFDFT_EINVAL, "masses must be > 0");
    c->masses.assign(m, m + c->nat);
    CK(cudaMemcpy(c->Md, m, c->nat * sizeof(double), cudaMemcpyHostToDevice));
    return OFDFT_OK;
}

ofdft_status ofdft_md_step(ofdft_ctx *c, const ofdft_md_params *mp, int nsteps, double *pos, double *vel,
                           double *F, ofdft_energy *E, ofdft_stats *stats)
{
    if (!c || !mp) return fail(c, OFDFT_EINVAL, "NULL argument");
    if (!(mp->dt_fs > 0.0) || !(mp->gtol > 0.0) || mp->maxit <= 0 || nsteps < 0)
        return fail(c, OFDFT_EINVAL, "bad MD parameters");
    cudaSetDevice(c->dev);
    const int nat = c->nat;
    ofdft_status s;
    if (pos && memcmp(pos, c->R.data(), 3 * nat * sizeof(double)) != 0) {
        c->R.assign(pos, pos + 3 * nat);
        CK(cudaMemcpyAsync(c->Rd, pos, 3 * nat * sizeof(double), cudaMemcpyHostToDevice, c->st));
        CK(cudaMemsetAsync(c->nh, 0, 4 * sizeof(double), c->st));
        s = update_ions(c);
        if (s != OFDFT_OK) return s;
        c->md_ready = false;
    }
    if (vel) CK(cudaMemcpyAsync(c->Vd, vel, 3 * nat * sizeof(double), cudaMemcpyHostToDevice, c->st));
    c->md_dt = mp->dt_fs * kFsAu;
    c->md_thermo = mp->T_kelvin > 0.0;
    c->md_kT = c->md_thermo ? mp->T_kelvin * kKbHa : 0.0;
    int ndof = 3 * nat - 3;
    double tau = (mp->tau_steps > 0 ? mp->tau_steps : 100.0) * c->md_dt;
    c->md_Q = c->md_thermo ? ndof * c->md_kT * tau * tau / (4.0 * kPi * kPi) : 1.0;
    ofdft_stats tot{};
    tot.status = OFDFT_OK;
    EvalScalars es;
    if (!c->md_ready) {
        ofdft_stats st{};
        s = run_minimize(c, mp->gtol, mp->maxit, st, es);
        tot.iterations += st.iterations;
        tot.evaluations += st.evaluations;
        tot.gnorm = st.gnorm;
        if (s != OFDFT_OK) {
            if (stats) *stats = tot;
            return s;
        }
        s = forces_now(c, es);
        if (s != OFDFT_OK) return s;
        size_t eb = c->precision == OFDFT_MIXED ? sizeof(float) : sizeof(double);
        CK(cudaMemcpyAsync(c->phiprev, c->phi, c->g.N * eb, cudaMemcpyDeviceToDevice, c->st));
        c->md_ready = true;
    }
    for (int step = 0; step < nsteps; ++step) {
        launch_md_a(nat, c->Md, c->Rd, c->Vd, c->Fd, c->md_dt, c->md_kT, c->md_Q, ndof, c->md_thermo, c->nh, c->st);
        c->launches++;
        s = update_ions(c);
        if (s != OFDFT_OK) return s;
        // density extrapolation phi0 = 2 phi_n - phi_{n-1}, renormalised by the minimiser
        if (ensure_part(c, 4096) != OFDFT_OK) return OFDFT_ENOMEM;
        if (c->precision == OFDFT_MIXED)
            launch_extrap<float>(c->g.N, (const float *)c->phi, (const float *)c->phiprev, (float *)c->phit, c->part, c->st);
        else
            launch_extrap<double>(c->g.N, (const double *)c->phi, (const double *)c->phiprev, (double *)c->phit, c->part, c->st);
        c->launches++;
        // rotate: phiprev <- phi, phi <- extrapolated
        std::swap(c->phiprev, c->phi);
        std::swap(c->phi, c->phit);
        ofdft_stats st{};
        s = run_minimize(c, mp->gtol, mp->maxit, st, es);
        tot.iterations += st.iterations;
        tot.evaluations += st.evaluations;
        tot.gnorm = st.gnorm;
        if (s != OFDFT_OK) {
            tot.status = s;
            if (stats) *stats = tot;
            return s;
        }
        s = forces_now(c, es);
        if (s != OFDFT_OK) return s;
        launch_md_b(nat, c->Md, c->Vd, c->Fd, c->md_dt, c->md_kT, c->md_Q, ndof, c->md_thermo, c->nh, c->st);
        c->launches++;
    }
    fill_energy(c, es, c->last);
    c->last_valid = true;
    if (pos) CK(cudaMemcpyAsync(pos, c->Rd, 3 * nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (vel) CK(cudaMemcpyAsync(vel, c->Vd, 3 * nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (F) CK(cudaMemcpyAsync(F, c->Fd, 3 * nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpy(c->R.data(), c->Rd, 3 * nat * sizeof(double), cudaMemcpyDeviceToHost));
    if (E) *E = c->last;
    if (stats) *stats = tot;
    return OFDFT_OK;
}

ofdft_status ofdft_md_state(ofdft_ctx *c, double *pos, double *vel)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    cudaSetDevice(c->dev);
    CK(cudaStreamSynchronize(c->st));
    if (pos) CK(cudaMemcpy(pos, c->Rd, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost));
    if (vel) CK(cudaMemcpy(vel, c->Vd, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost));
    return OFDFT_OK;
}

ofdft_status ofdft_md_conserved(ofdft_ctx *c, double *H)
{
    if (!c || !H) return fail(c, OFDFT_EINVAL, "NULL argument");
    if (!c->last_valid) return fail(c, OFDFT_EINVAL, "no MD step has run");
    double nh[4];
    CK(cudaMemcpy(nh, c->nh, sizeof(nh), cudaMemcpyDeviceToHost));
    int ndof = 3 * c->nat - 3;
    *H = nh[2] + c->last.F_tot + 0.5 * c->md_Q * nh[0] * nh[0] + ndof * c->md_kT * nh[1];
    return OFDFT_OK;
}

ofdft_status ofdft_sizes(ofdft_ctx *c, long long *N, int *nat)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    if (N) *N = c->g.N;
    if (nat) *nat = c->nat;
    return OFDFT_OK;
}

ofdft_status ofdft_timer_select(ofdft_ctx *c, int id)
{
    if (!c || id < 0 || id > 7) return fail(c, OFDFT_EINVAL, "bad timer id");
    c->timer_id = id;
    c->tev_used = 0;
    return OFDFT_OK;
}

ofdft_status ofdft_timer_read(ofdft_ctx *c, double *total_ms, long long *launches, int reset)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    cudaSetDevice(c->dev);
    CK(cudaStreamSynchronize(c->st));
    double tot = 0.0;
    for (size_t i = 0; i + 1 < c->tev_used; i += 2) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, c->tev[i], c->tev[i + 1]));
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (long long)(c->tev_used / 2);
    if (reset) c->tev_used = 0;
    return OFDFT_OK;
}

long long ofdft_kernel_launches(ofdft_ctx *c) { return c ? c->launches : 0; }

const char *ofdft_last_error(ofdft_ctx *c) { return c ? c->err.c_str() : g_setup_error.c_str(); }

ofdft_status ofdft_tfunc_eval(long long n, const double *t, double *out)
{
    if (n < 0 || (n > 0 && (!t || !out))) return OFDFT_EINVAL;
    const std::vector<double> &tab = tfunc_table_host();
    for (long long i = 0; i < n; ++i) {
        if (!(t[i] > 0.0)) return OFDFT_EINVAL;
        tfunc_eval<double>(tab.data(), t[i], out + 8 * i);
    }
    return OFDFT_OK;
}

void ofdft_destroy(ofdft_ctx *c) { free_ctx(c); }

}  // extern "C"
