// C ABI of libofdft (include/ofdft.h): context, evaluation pipeline, CG
// minimiser, forces, pressure and MD driver.
//
// A minimisation runs entirely on the device: the vector kernels read their
// scalars from a CgState in device memory, single-thread controller kernels
// update it, and the two loops (CG iterations, line-search trials) are CUDA
// graph conditional WHILE nodes, so one graph launch performs a whole
// minimisation without host synchronisation.  With OFDFT_DEBUG_SYNC=1 or an
// active kernel timer the same kernel sequence is driven from the host.
#include <math.h>

#include <cmath>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <tuple>
#include <mutex>
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

thread_local std::string g_setup_error;   // setup errors (no context yet), per thread

// Working fields of one precision.
struct FieldSet {
    bool valid = false;
    void *phi = nullptr, *phit = nullptr, *dhat = nullptr, *g = nullptr, *gprev = nullptr,
         *d = nullptr, *v = nullptr, *vt = nullptr, *vpart = nullptr;
    void *spec = nullptr;      // four half spectra, one allocation
    size_t spec_stride = 0;    // elements between spectra
    void *vext = nullptr, *tab = nullptr;
    void *tw[3] = {nullptr, nullptr, nullptr};
    FftAxis ax[3];
    CgState *cs = nullptr;     // device CG state
    cudaGraphExec_t graph = nullptr;
    GridInfo gt{};             // the grid with this set's launch shapes (ofdft_autotune)
};

}  // namespace

struct ofdft_ctx {
    int dev = 0;
    cudaStream_t st = nullptr, cap2 = nullptr;
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
    FieldSet f[2];              // [0] FP64 (always), [1] FP32 (mixed contexts)
    double *phiprev = nullptr;  // FP64 density history for MD extrapolation
    double *part = nullptr;     // reduction partials, fixed size
    size_t part_len = 0;
    double *scal = nullptr;     // device scalars outside a minimisation
    double *scal_h = nullptr;   // pinned host copy
    CgState *cfg_h[2] = {nullptr, nullptr};   // pinned CG configuration per field set
    CgState *st_h[2] = {nullptr, nullptr};    // pinned final CG state per field set
    cudaEvent_t done_ev = nullptr;             // end of the minimisation in flight
    bool pending = false, pend_graph = false;
    // ions
    double *Rd = nullptr, *Zd = nullptr, *Fd = nullptr, *Vd = nullptr, *Md = nullptr, *nh = nullptr;
    double2 *px = nullptr, *py = nullptr, *pz = nullptr;
    PhaseTablesDD pdd = {nullptr, nullptr, nullptr, nullptr};   // double-float copies (one allocation at xT)
    double *fpart = nullptr;
    size_t fpart_len = 0;
    // Ewald
    double *Gv = nullptr, *wG = nullptr, *eion = nullptr, *ewF = nullptr, *ewpart = nullptr;
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
    bool debug_sync = false;    // OFDFT_DEBUG_SYNC=1: check every launch, no graphs
    bool use_graphs = true;     // OFDFT_NO_GRAPHS=1: host-driven loops
    // fork/join of a GGA evaluation: two auxiliary streams (the Hartree
    // chain; the second derivative pass of a pair) and the events between
    // them and the evaluation's stream
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t fj[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // kernel timer (diagnostics)
    int timer_id = 0;
    std::vector<cudaEvent_t> tev;
    size_t tev_used = 0;
    // batched form: this context's identity and launch-shape epoch, and the
    // executable graph of the last batch it led (one branch per instance)
    unsigned long long uid = 0;
    unsigned shape_epoch = 0;
    std::vector<unsigned long long> batch_key;
    cudaGraphExec_t batch_exec = nullptr;
};

namespace {

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e_), #call);     \
    } while (0)

ofdft_status fail(ofdft_ctx *c, ofdft_status s, const char *msg, const char *where = nullptr)
{
    std::string m = msg ? msg : "error";
    if (where) m += std::string(" at ") + where;
    if (c) c->err = m;
    else g_setup_error = m;
    return s;
}

// With OFDFT_DEBUG_SYNC=1 every launch is followed by a stream synchronisation
// and an error check that names the kernel.
ofdft_status dbg(ofdft_ctx *c, const char *what)
{
    if (!c->debug_sync) return OFDFT_OK;
    cudaError_t e = cudaPeekAtLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), what);
    }
    return OFDFT_OK;
}

#define DBG(name)                                              \
    do {                                                       \
        if (dbg(c, name) != OFDFT_OK) return OFDFT_EDEVICE;    \
    } while (0)

bool smooth_even(int n)
{
    if (n < 8 || n > 512 || (n & 1)) return false;
    int m = n;
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}


template <typename T> ofdft_status upload_twiddles(ofdft_ctx *c, FieldSet &f, int axis, int n)
{
    std::vector<cplx<T>> w(n);
    for (int m = 0; m < n; ++m) {
        long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)n;
        w[m].x = (T)cosl(ang);
        w[m].y = (T)sinl(ang);
    }
    // FP64 sets append the same twiddles as double-float pairs (ff::cf2)
    std::vector<float> wf;
    if (sizeof(T) == 8) {
        wf.resize(4 * (size_t)n);
        for (int m = 0; m < n; ++m) {
            long double ang = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)n;
            long double cv = cosl(ang), sv = sinl(ang);
            float ch = (float)cv, sh = (float)sv;
            wf[4 * m] = ch;
            wf[4 * m + 1] = (float)(cv - (long double)ch);
            wf[4 * m + 2] = sh;
            wf[4 * m + 3] = (float)(sv - (long double)sh);
        }
    }
    const size_t nb = n * sizeof(cplx<T>), nbf = wf.size() * sizeof(float);
    CK(cudaMallocAsync((void **)&f.tw[axis], nb + nbf, c->st));
    CK(cudaMemcpyAsync(f.tw[axis], w.data(), nb, cudaMemcpyHostToDevice, c->st));
    if (nbf) CK(cudaMemcpyAsync((char *)f.tw[axis] + nb, wf.data(), nbf, cudaMemcpyHostToDevice, c->st));
    // FP64 z passes: power-of-two radices up to 4 (shorter double-float
    // butterfly chains between the barriers of the fused z kernels)
    f.ax[axis] = fft_axis(n, f.tw[axis], (sizeof(T) == 8 && axis == 2) ? 4 : 8);
    f.ax[axis].twf = nbf ? (const void *)((const char *)f.tw[axis] + nb) : nullptr;
    return OFDFT_OK;
}

ofdft_status sync_read(ofdft_ctx *c, int n)
{
    CK(cudaMemcpyAsync(c->scal_h, c->scal, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaGetLastError());
    return OFDFT_OK;
}

enum TimerId { TM_PW = 1, TM_DLINE = 2, TM_Y = 4, TM_ZFWD = 5, TM_ZFINAL = 6, TM_XHL = 7 };

// Event pair around a launch of the selected kernel class (host-driven mode
// only).  The selection's bit 8 restricts it to the FP32 launches, bit 16 to
// the FP64 ones.
struct TimerScope {
    ofdft_ctx *c;
    bool on;
    TimerScope(ofdft_ctx *c_, int id, bool f32)
        : c(c_), on((c_->timer_id & 7) == id && !((c_->timer_id & 8) && !f32) && !((c_->timer_id & 16) && f32))
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

// ------------------------------------------------------------ evaluation
// Sums written by one evaluation (18 doubles): [0] E_H [1] E_loc [2] P_loc,
// [3..8] GGA pointwise sums, [9..17] final-stage sums (F_s, TS, F_xc,
// n df/dn - f, -, n(v_xc - eps), phi^2 v, phi^2, dE/dtheta).
struct EvalScalars {
    double EH, Eloc, Ploc, FS, TS, FXC, PS, WG, PXC, PHI2V, PHI2, DTH;
};

EvalScalars unpack_sums(const double *h, bool fttf)
{
    EvalScalars es;
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
    return es;
}

int eval_kernel_count(const ofdft_ctx *c) { return c->fp.kind == 0 ? 6 : 11; }

// Enqueue one energy + potential evaluation at ph (or, with phi0 and dh, at the
// trial phi0 cos + dh sin written into ph; angles from csd (two T values in
// device memory) if given).  Sums go to sums[0..17].  With keep_nG, n(G) is
// left in the second spectrum (forces, stress).  With spart (FP64 GGA sets),
// the pointwise stage also writes the gradient stress sums: spart holds 12
// partial rows of *nbg_out columns.  No synchronisation.
//
// ftTF:  zfwd (n, R2C z) -> y -> x [Hartree, LPP, energies, v_HL(G), x^-1]
//        -> y^-1 -> zfinal [C2R z, pointwise, potential, sums].
// GGA:   the same Hartree path, and the gradient and divergence one axis at
//        a time (the derivative along axis j needs transforms along j only):
//        zfwd also writes d_z n; dline x, y: d_x n, d_y n (second to fourth
//        spectra, used as real fields); pointwise: v_part and U_j over the
//        derivatives; dline x, y: d_x U_x + d_y U_y into vout; zfinal_gga:
//        v = v_HL - d_z U_z + v_part - (d_x U_x + d_y U_y), sums.
template <typename T>
ofdft_status enqueue_eval(ofdft_ctx *c, FieldSet &f, T *ph, const T *phi0, const T *dh, double cth,
                          double sth, const void *csd, T *vout, bool keep_nG, double *sums,
                          double *spart = nullptr, int *nbg_out = nullptr)
{
    const GridInfo &g = f.gt;
    const FftAxis &ax = f.ax[0], &ay = f.ax[1], &az = f.ax[2];
    cudaStream_t st = c->st;
    typedef cplx<T> C;
    C *s0 = (C *)f.spec;
    const long long fs = (long long)f.spec_stride;
    C *s1 = s0 + fs, *s2 = s1 + fs, *s3 = s2 + fs;
    T *d0 = (T *)s1, *d1 = (T *)s2, *d2 = (T *)s3;   // real fields of N values (a spectrum holds 2 NH >= N)
    const C *vext = (const C *)f.vext;
    const T *tab = (const T *)f.tab;
    const bool fttf = c->fp.kind == 0;
    const int nbx = xpass_blocks(g);
    const long long npairs = (long long)g.nx * g.ny / 2;
    double *pA = c->part, *pB = pA + 3 * nbx, *pC = pB + 6 * npairs;
    {
        TimerScope ts(c, TM_ZFWD, sizeof(T) == 4);
        T *dz = fttf ? nullptr : d2;
        if (phi0) launch_zfwd<T>(g, az, 2, nullptr, phi0, dh, (T)cth, (T)sth, csd, ph, s0, st, dz);
        else launch_zfwd<T>(g, az, 1, nullptr, ph, nullptr, T(0), T(0), nullptr, nullptr, s0, st, dz);
    }
    DBG("k_zfwd");
    // GGA: the Hartree chain (y, x, y^-1 on the first spectrum) needs only
    // zfwd's spectrum and the gradient chain only phi and d_z n, so the
    // chain runs on aux[0] beside the derivative passes and the pointwise
    // stage; the two derivative passes of each pair run side by side
    // (aux[1]).  Timers and per-launch checks keep one stream.
    const bool fork = !fttf && c->aux[0] && c->timer_id == 0 && !c->debug_sync;
    cudaStream_t sh = st;   // stream of the Hartree chain
    if (fork) {
        CK(cudaEventRecord(c->fj[0], st));
        CK(cudaStreamWaitEvent(c->aux[0], c->fj[0], 0));
        CK(cudaStreamWaitEvent(c->aux[1], c->fj[0], 0));
        sh = c->aux[0];
    }
    {
        TimerScope ts(c, TM_Y, sizeof(T) == 4);
        launch_ypass<T>(g, ay, false, s0, 1, fs, sh);
    }
    DBG("k_ypass fwd");
    {
        TimerScope ts(c, TM_XHL, sizeof(T) == 4);
        launch_xhl<T>(g, ax, s0, vext, (keep_nG && fttf) ? s1 : nullptr, 1, pA, sh);
    }
    DBG("k_xhl");
    {
        TimerScope ts(c, TM_Y, sizeof(T) == 4);
        launch_ypass<T>(g, ay, true, s0, 1, fs, sh);
    }
    DBG("k_ypass inv");
    if (fork) CK(cudaEventRecord(c->fj[1], sh));
    int nbz, nbg = 0;   // blocks of the z passes (zfinal) and of the pointwise stage: their partial sums
    if (fttf) {
        TimerScope ts(c, TM_ZFINAL, sizeof(T) == 4);
        nbz = launch_zfinal<T>(g, az, true, s0, nullptr, ph, phi0, dh, (T)cth, (T)sth, csd, (T)c->T,
                               c->fp, tab, c->xc, vout, pC, st);
    } else {
        cudaStream_t s2nd = fork ? c->aux[1] : st;   // stream of each pair's second pass
        {
            TimerScope ts(c, TM_DLINE, sizeof(T) == 4);
            launch_dline<T>(g, ax, 0, 0, 0, ph, d0, st);
        }
        {
            TimerScope ts(c, TM_DLINE, sizeof(T) == 4);
            launch_dline<T>(g, ay, 1, 0, 0, ph, d1, s2nd);
        }
        if (fork) {
            CK(cudaEventRecord(c->fj[2], s2nd));
            CK(cudaStreamWaitEvent(st, c->fj[2], 0));
        }
        DBG("k_dline (grad n)");
        {
            TimerScope ts(c, TM_PW, sizeof(T) == 4);
            if (spart) {
                pB = spart;
                nbg = launch_pw<T>(g, d0, d1, d2, ph, (T)c->T, c->fp, tab, c->xc, (T *)f.vpart, pB, true, st);
                if (nbg_out) *nbg_out = nbg;
            } else {
                nbg = launch_pw<T>(g, d0, d1, d2, ph, (T)c->T, c->fp, tab, c->xc, (T *)f.vpart, pB, false, st);
            }
        }
        DBG("k_pw");
        if (fork) {
            CK(cudaEventRecord(c->fj[3], st));
            CK(cudaStreamWaitEvent(s2nd, c->fj[3], 0));
        }
        // d_y U_y into vout, d_x U_x in place over U_x (d0); the final z pass
        // subtracts both
        {
            TimerScope ts(c, TM_DLINE, sizeof(T) == 4);
            launch_dline<T>(g, ay, 1, 1, 0, d1, vout, st);
        }
        {
            TimerScope ts(c, TM_DLINE, sizeof(T) == 4);
            launch_dline<T>(g, ax, 0, 1, 0, d0, d0, s2nd);
        }
        if (fork) {
            CK(cudaEventRecord(c->fj[4], s2nd));
            CK(cudaStreamWaitEvent(st, c->fj[4], 0));
            CK(cudaStreamWaitEvent(st, c->fj[1], 0));
        }
        DBG("k_dline (div W)");
        TimerScope ts(c, TM_ZFINAL, sizeof(T) == 4);
        nbz = launch_zfinal_gga<T>(g, az, s0, d2, (const T *)f.vpart, vout, d0, ph, phi0, dh, (T)cth, (T)sth,
                                   csd, vout, pC, st);
    }
    DBG("k_zfinal");
    launch_reduce_eval(pA, nbx, pB, nbg, pC, nbz, !fttf, sums, st);
    DBG("k_reduce_eval");
    c->launches += eval_kernel_count(c);
    if (keep_nG && !fttf) {
        // n(G) for forces and stress: forward z, y, x of n into the second spectrum
        launch_zfwd<T>(g, az, 1, nullptr, ph, nullptr, T(0), T(0), nullptr, nullptr, s1, st);
        launch_ypass<T>(g, ay, false, s1, 1, fs, st);
        launch_xhl<T>(g, ax, s1, vext, s1, 0, pA, st);
        c->launches += 3;
        DBG("n(G)");
    }
    return OFDFT_OK;
}

// One evaluation outside a minimisation, read back to the host.
template <typename T>
ofdft_status evaluate(ofdft_ctx *c, FieldSet &f, T *ph, T *vout, bool keep_nG, EvalScalars &es)
{
    ofdft_status s = enqueue_eval<T>(c, f, ph, nullptr, nullptr, 1.0, 0.0, nullptr, vout, keep_nG, c->scal);
    if (s != OFDFT_OK) return s;
    if (sync_read(c, 18) != OFDFT_OK) return OFDFT_EDEVICE;
    es = unpack_sums(c->scal_h, c->fp.kind == 0);
    double chk = es.EH + es.Eloc + es.FS + es.FXC + es.PHI2V;
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
    // G -> 0 limit of Omega w(G) + 4 pi Z/G^2 per ion: pi Z rc^2 (Gaussian),
    // 2 pi Z rc^2 - (4 pi/3) A rc^3 (Eq. (E4A): -A inside rc, -Z/r outside)
    const double rc = c->g.rc;
    double zs = 0.0;
    for (int i = 0; i < c->nat; ++i)
        zs += c->g.lpp ? 2.0 * kPi * c->Z[i] * rc * rc - (4.0 / 3.0) * kPi * c->g.ha_A * rc * rc * rc
                       : kPi * c->Z[i] * rc * rc;
    E.E_alphaZ = c->Ne * zs / om;
    E.P_s = (dV * es.PS + (4.0 / 3.0) * dV * es.WG) / om;
    E.P_xc = dV * es.PXC / om;
    E.P_H = es.EH / (3.0 * om);
    E.P_loc = es.Ploc;
    E.P_ion = c->E_ion / (3.0 * om);
    E.P = E.P_s + E.P_xc + E.P_H + E.P_loc + E.P_ion;
}

// ---------------------------------------------------------- ions & Ewald
EwCell ew_cell(const GridInfo &g)
{
    EwCell e;
    for (int k = 0; k < 9; ++k) {
        e.a[k] = g.Am[k];
        e.ai[k] = g.Ainv[k];
    }
    e.tri = g.tri;
    return e;
}

ofdft_status setup_ewald(ofdft_ctx *c)
{
    const GridInfo &g = c->g;
    double om = g.omega;
    c->ew_alpha = 1.2 * sqrt(kPi) * pow((double)c->nat / (om * om), 1.0 / 6.0);
    c->ew_rcut = 6.3 / c->ew_alpha;
    // lattice planes normal to b_j are h_j = 2 pi/|b_j| apart; |a_j| bounds G.a_j/2 pi
    double h[3], La[3];
    for (int j = 0; j < 3; ++j) {
        const double *b = g.Bm + 3 * j, *a = g.Am + 3 * j;
        h[j] = 2.0 * kPi / sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        La[j] = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    }
    if (!g.tri) {
        h[0] = La[0] = g.Lx;
        h[1] = La[1] = g.Ly;
        h[2] = La[2] = g.Lz;
    }
    c->ew_nimg = make_int3((int)ceil(c->ew_rcut / h[0] + 0.5), (int)ceil(c->ew_rcut / h[1] + 0.5),
                           (int)ceil(c->ew_rcut / h[2] + 0.5));
    double gcut = 2.0 * c->ew_alpha * 6.3;
    int km[3];
    for (int a = 0; a < 3; ++a) km[a] = (int)ceil(gcut * La[a] / (2.0 * kPi));
    std::vector<double> Gv, wG;
    const double *B = g.Bm;
    for (int i = -km[0]; i <= km[0]; ++i)
        for (int j = -km[1]; j <= km[1]; ++j)
            for (int k = -km[2]; k <= km[2]; ++k) {
                double gx = 2 * kPi * i / g.Lx, gy = 2 * kPi * j / g.Ly, gz = 2 * kPi * k / g.Lz;
                if (g.tri) {
                    gx = i * B[0] + j * B[3] + k * B[6];
                    gy = i * B[1] + j * B[4] + k * B[7];
                    gz = i * B[2] + j * B[5] + k * B[8];
                }
                double g2 = gx * gx + gy * gy + gz * gz;
                if (g2 == 0.0 || g2 >= gcut * gcut) continue;
                Gv.push_back(gx);
                Gv.push_back(gy);
                Gv.push_back(gz);
                wG.push_back(2.0 * kPi / om * exp(-g2 / (4.0 * c->ew_alpha * c->ew_alpha)) / g2);
            }
    c->nGe = (int)wG.size();
    int nb = (c->nGe + 255) / 256;
    CK(cudaMallocAsync((void **)&c->Gv, std::max<size_t>(1, Gv.size()) * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->wG, std::max<size_t>(1, wG.size()) * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->Se, std::max(1, c->nGe) * sizeof(double2), c->st));
    CK(cudaMallocAsync((void **)&c->ewpart, std::max(1, nb) * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->eion, c->nat * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->ewF, 3 * c->nat * sizeof(double), c->st));
    if (!Gv.empty()) {
        CK(cudaMemcpyAsync(c->Gv, Gv.data(), Gv.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
        CK(cudaMemcpyAsync(c->wG, wG.data(), wG.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    }
    return OFDFT_OK;
}

// Recompute v_ext(G) (every field set) and the Ewald energy and forces from Rd.
ofdft_status update_ions(ofdft_ctx *c)
{
    const GridInfo &g = c->g;
    cudaStream_t st = c->st;
    const PhaseTablesDD *dd = g.dd ? &c->pdd : nullptr;
    launch_phases(g, c->nat, c->Rd, c->px, c->py, c->pz, dd, st);
    launch_vext(g, c->nat, c->Zd, c->px, c->py, c->pz, dd, (double2 *)c->f[0].vext, st);
    if (c->f[1].valid)
        launch_convert<double, float>(((g.lpp || g.tri) ? 4 : 2) * g.NH, (const double *)c->f[0].vext, (float *)c->f[1].vext,
                                      st);
    launch_ewald_real(c->nat, c->Rd, c->Zd, ew_cell(g), c->ew_alpha, c->ew_rcut, c->ew_nimg, c->eion, c->ewF, st);
    int nb = launch_ewald_recip(c->nat, c->Rd, c->Zd, c->nGe, c->Gv, c->wG, c->Se, c->ewpart, c->ewF, st);
    c->launches += 5 + (c->f[1].valid ? 1 : 0);
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
// Kernel sequence of a minimisation on field set f; with use_cond the
// controllers drive the graph's conditional handles.
template <typename T>
ofdft_status enqueue_prologue(ofdft_ctx *c, FieldSet &f, cudaGraphConditionalHandle outer, int use_cond)
{
    const long long N = c->g.N;
    cudaStream_t st = c->st;
    CgState *s = f.cs;
    int nb = launch_sumsq<T>(N, (const T *)f.phi, c->part, st);
    launch_reduce(c->part, nb, 1, s->rn, st);
    launch_ctl_norm(s, st);
    launch_scale<T>(N, (T *)f.phi, 1.0, &s->scale, st);
    c->launches += 4;
    DBG("normalise");
    ofdft_status r = enqueue_eval<T>(c, f, (T *)f.phi, nullptr, nullptr, 1.0, 0.0, nullptr, (T *)f.v, false, s->ev);
    if (r != OFDFT_OK) return r;
    launch_ctl_init(s, st);
    nb = launch_cg_grad<T>(N, (const T *)f.phi, (const T *)f.v, 0.0, &s->mu, (T *)f.g, nullptr, c->part, st);
    launch_reduce(c->part, nb, 2, s->rg, st);
    launch_ctl_grad(s, 1, outer, use_cond, st);
    c->launches += 4;
    DBG("cg prologue");
    return OFDFT_OK;
}

template <typename T>
ofdft_status enqueue_direction(ofdft_ctx *c, FieldSet &f, cudaGraphConditionalHandle ls, int use_cond)
{
    const long long N = c->g.N;
    cudaStream_t st = c->st;
    CgState *s = f.cs;
    int nb = launch_cg_dir<T>(N, (const T *)f.g, (T *)f.d, 0.0, &s->beta, (const T *)f.phi, c->part, st);
    launch_reduce(c->part, nb, 5, s->rd, st);
    launch_ctl_dir(s, st);
    nb = launch_cg_dhat<T>(N, (const T *)f.g, (T *)f.d, (const T *)f.phi, (const T *)f.v, 0.0, 0.0, 0,
                           s->c12r, (T *)f.dhat, c->part, st);
    launch_reduce(c->part, nb, 1, s->rh, st);
    launch_ctl_dhat(s, ls, use_cond, st);
    c->launches += 6;
    DBG("cg direction");
    return OFDFT_OK;
}

template <typename T>
ofdft_status enqueue_trial(ofdft_ctx *c, FieldSet &f, cudaGraphConditionalHandle ls, int use_cond)
{
    CgState *s = f.cs;
    const void *cs = sizeof(T) == 8 ? (const void *)s->cs : (const void *)s->csf;   // angle in T
    ofdft_status r = enqueue_eval<T>(c, f, (T *)f.phit, (const T *)f.phi, (const T *)f.dhat, 1.0, 0.0, cs,
                                     (T *)f.vt, false, s->ev);
    if (r != OFDFT_OK) return r;
    launch_ctl_ls(s, ls, use_cond, c->st);
    c->launches += 1;
    DBG("line search");
    return OFDFT_OK;
}

template <typename T>
ofdft_status enqueue_update(ofdft_ctx *c, FieldSet &f, cudaGraphConditionalHandle outer, int use_cond)
{
    const long long N = c->g.N;
    cudaStream_t st = c->st;
    CgState *s = f.cs;
    int nb = launch_cg_update<T>(N, &s->accepted, (T *)f.phi, (const T *)f.phit, (T *)f.v, (const T *)f.vt,
                                 &s->mu, (T *)f.g, (T *)f.gprev, c->part, st);
    launch_reduce(c->part, nb, 2, s->rg, st);
    launch_ctl_grad(s, 0, outer, use_cond, st);
    c->launches += 3;
    DBG("cg update");
    return OFDFT_OK;
}

// Add a WHILE conditional node at the capture position of `stream`; returns
// its body graph.  The handle must belong to the graph being captured.
ofdft_status add_while(ofdft_ctx *c, cudaStream_t stream, cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaStreamCaptureStatus cst;
    cudaGraph_t gr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(stream, &cst, nullptr, &gr, &deps, &ed, &nd));
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, gr, deps, ed, nd, &p));
    *body = p.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return OFDFT_OK;
}

// Fill the body of a minimisation's outer WHILE node (field set f, outer
// handle):  direction; WHILE(ls) { trial }; update.  The bodies of the two
// loops are captured one after the other into the graphs their nodes own.
template <typename T>
ofdft_status capture_body(ofdft_ctx *c, FieldSet &f, cudaGraphConditionalHandle outer, cudaGraph_t body)
{
    cudaStream_t cs = c->cap2;
    cudaGraphConditionalHandle ls = 0;
    cudaGraph_t ls_body = nullptr;
    ofdft_status r = OFDFT_OK;
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaGraphConditionalHandleCreate(&ls, body, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) r = fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "graph handle");
    if (r == OFDFT_OK) r = enqueue_direction<T>(c, f, ls, 1);
    if (r == OFDFT_OK) r = add_while(c, cs, ls, &ls_body);
    if (r == OFDFT_OK) r = enqueue_update<T>(c, f, outer, 1);
    e = cudaStreamEndCapture(cs, &body);
    if (r != OFDFT_OK) return r;
    if (e != cudaSuccess) return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "graph capture (outer body)");

    CK(cudaStreamBeginCaptureToGraph(cs, ls_body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    r = enqueue_trial<T>(c, f, ls, 1);
    e = cudaStreamEndCapture(cs, &ls_body);
    if (r != OFDFT_OK) return r;
    if (e != cudaSuccess) return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "graph capture (line search)");
    return OFDFT_OK;
}

// Enqueue (on the capturing stream c->cap2) the prologue of field set f's
// minimisation and its outer WHILE node, whose handle is created on graph
// gr; returns the handle and the node's body graph.
template <typename T>
ofdft_status capture_outer(ofdft_ctx *c, FieldSet &f, cudaGraph_t gr, cudaGraphConditionalHandle *outer,
                           cudaGraph_t *body)
{
    cudaError_t e = cudaGraphConditionalHandleCreate(outer, gr, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "graph handle");
    ofdft_status r = enqueue_prologue<T>(c, f, *outer, 1);
    if (r == OFDFT_OK) r = add_while(c, c->cap2, *outer, body);
    return r;
}

// Capture the whole minimisation of field set f into a graph:
//   prologue; WHILE(outer) { direction; WHILE(ls) { trial }; update }
// Capture runs on the private stream cap2 (the context's stream may be the
// legacy stream, which cannot be captured).
template <typename T> ofdft_status capture_graph(ofdft_ctx *c, FieldSet &f, cudaGraph_t *whole)
{
    cudaStream_t cs = c->cap2;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    cudaStreamCaptureStatus cst;
    cudaGraph_t gr = nullptr;
    cudaGraphConditionalHandle outer = 0;
    cudaGraph_t body = nullptr;
    ofdft_status r = OFDFT_OK;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &gr, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) r = fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "graph capture info");
    if (r == OFDFT_OK) r = capture_outer<T>(c, f, gr, &outer, &body);
    e = cudaStreamEndCapture(cs, whole);
    if (r != OFDFT_OK) return r;
    if (e != cudaSuccess) return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "graph capture");
    return capture_body<T>(c, f, outer, body);
}

template <typename T> ofdft_status build_graph(ofdft_ctx *c, FieldSet &f)
{
    cudaStream_t user = c->st;
    long long before = c->launches;
    const bool dbg_saved = c->debug_sync;
    c->st = c->cap2;
    c->debug_sync = false;
    cudaGraph_t whole = nullptr;
    ofdft_status r = capture_graph<T>(c, f, &whole);
    c->st = user;
    c->debug_sync = dbg_saved;
    c->launches = before;
    if (r == OFDFT_OK) {
        cudaError_t e = cudaGraphInstantiate(&f.graph, whole, 0);
        if (e != cudaSuccess) {
            f.graph = nullptr;
            r = fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "graph instantiation");
        }
    }
    if (whole) cudaGraphDestroy(whole);
    return r;
}

// Field set k's CG configuration is staged in pinned memory (one buffer per
// set, so the two copies of a mixed-precision minimisation never race).
ofdft_status write_config(ofdft_ctx *c, int k, double gtol, int maxit, int stagnate, cudaStream_t on = nullptr)
{
    CgState *h = c->cfg_h[k];
    memset(h, 0, sizeof(CgState));
    h->gtol = gtol;
    // the FP32 stage of a mixed minimisation hands over to FP64 once
    // ||g|| < 1e-5 (or earlier, when it stalls at the single-precision floor)
    h->switch_g = stagnate ? std::max(1e-5, 10.0 * gtol) : 0.0;
    h->dV = c->g.dV;
    h->ls_tol = 0.1;
    h->eoff = c->fp.kind == 0 ? 9 : 3;
    // line-search energy test: rounding allowance of the energy sums
    h->e_tol = k == 0 ? 1e-11 : 1e-5;
    h->theta0 = 0.05;
    h->Ne = c->Ne;
    h->maxit = maxit;
    h->max_ls = 20;
    h->stagnate = stagnate;
    h->status = OFDFT_OK;
    CK(cudaMemcpyAsync(c->f[k].cs, h, sizeof(CgState), cudaMemcpyHostToDevice, on ? on : c->st));
    return OFDFT_OK;
}

ofdft_status read_state(ofdft_ctx *c, int k)
{
    CK(cudaMemcpyAsync(c->st_h[k], c->f[k].cs, sizeof(CgState), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaGetLastError());
    return OFDFT_OK;
}

bool graphs_on(const ofdft_ctx *c) { return c->use_graphs && !c->debug_sync && c->timer_id == 0; }

// Enqueue the minimisation of field set k as one graph launch (phi already
// holds the start) and the copy of its final CG state to st_h[k].
template <typename T>
ofdft_status enqueue_minimize_graph(ofdft_ctx *c, int k, double gtol, int maxit, int stagnate)
{
    FieldSet &f = c->f[k];
    if (write_config(c, k, gtol, maxit, stagnate) != OFDFT_OK) return OFDFT_EDEVICE;
    if (!f.graph) {
        ofdft_status r = build_graph<T>(c, f);
        if (r != OFDFT_OK) return r;
    }
    CK(cudaGraphLaunch(f.graph, c->st));
    CK(cudaMemcpyAsync(c->st_h[k], f.cs, sizeof(CgState), cudaMemcpyDeviceToHost, c->st));
    return OFDFT_OK;
}

// The same kernel sequence driven from the host (debugging, kernel timers).
template <typename T>
ofdft_status minimize_host(ofdft_ctx *c, int k, double gtol, int maxit, int stagnate)
{
    FieldSet &f = c->f[k];
    if (write_config(c, k, gtol, maxit, stagnate) != OFDFT_OK) return OFDFT_EDEVICE;
    cudaGraphConditionalHandle none = 0;
    ofdft_status r = enqueue_prologue<T>(c, f, none, 0);
    if (r != OFDFT_OK) return r;
    if (read_state(c, k) != OFDFT_OK) return OFDFT_EDEVICE;
    while (!c->st_h[k]->done) {
        if ((r = enqueue_direction<T>(c, f, none, 0)) != OFDFT_OK) return r;
        do {
            if ((r = enqueue_trial<T>(c, f, none, 0)) != OFDFT_OK) return r;
            if (read_state(c, k) != OFDFT_OK) return OFDFT_EDEVICE;
        } while (c->st_h[k]->ls_active);
        if ((r = enqueue_update<T>(c, f, none, 0)) != OFDFT_OK) return r;
        if (read_state(c, k) != OFDFT_OK) return OFDFT_EDEVICE;
    }
    return OFDFT_OK;
}

// Start a minimisation.  With graphs the whole solve (both precisions of a
// mixed context: FP32 CG until converged or stalled at the single-precision
// floor, then FP64 CG from there to gtol) is enqueued on the context's
// stream and this returns at once; otherwise it runs to completion here.
ofdft_status minimize_start(ofdft_ctx *c, double gtol, int maxit)
{
    if (c->pending) return fail(c, OFDFT_EBUSY, "a minimisation is already in flight");
    const bool mixed = c->precision == OFDFT_MIXED;
    const bool graphs = graphs_on(c);
    ofdft_status s = OFDFT_OK;
    c->pend_graph = graphs;
    if (mixed) {
        launch_convert<double, float>(c->g.N, (const double *)c->f[0].phi, (float *)c->f[1].phi, c->st);
        c->launches++;
        s = graphs ? enqueue_minimize_graph<float>(c, 1, gtol, maxit, kStagnateIts)
                   : minimize_host<float>(c, 1, gtol, maxit, kStagnateIts);
        if (s != OFDFT_OK) return s;
        launch_convert<float, double>(c->g.N, (const float *)c->f[1].phi, (double *)c->f[0].phi, c->st);
        c->launches++;
    }
    s = graphs ? enqueue_minimize_graph<double>(c, 0, gtol, maxit, 0) : minimize_host<double>(c, 0, gtol, maxit, 0);
    if (s != OFDFT_OK) return s;
    CK(cudaEventRecord(c->done_ev, c->st));
    c->pending = true;
    return OFDFT_OK;
}

// Launches of one graph-driven minimisation: prologue, per outer iteration
// (direction + update), per line-search trial (evaluation + controller).
long long graph_launches(const ofdft_ctx *c, const CgState &h)
{
    return 8 + eval_kernel_count(c) + (long long)h.nouter * 9 +
           (long long)(h.nevals - 1) * (eval_kernel_count(c) + 1);
}

ofdft_status finish_minimize(ofdft_ctx *c, bool graph, ofdft_stats &stats, EvalScalars &es);

// Wait for the minimisation started last; fill stats and the energies.
ofdft_status minimize_wait(ofdft_ctx *c, ofdft_stats &stats, EvalScalars &es)
{
    stats = ofdft_stats{};
    if (!c->pending) return fail(c, OFDFT_EINVAL, "no minimisation in flight");
    c->pending = false;
    CK(cudaEventSynchronize(c->done_ev));
    CK(cudaGetLastError());
    return finish_minimize(c, c->pend_graph, stats, es);
}

// Statistics and energies of a finished minimisation from the final CG
// states in st_h (graph: count the launches the graph made).
ofdft_status finish_minimize(ofdft_ctx *c, bool graph, ofdft_stats &stats, EvalScalars &es)
{
    stats = ofdft_stats{};
    const bool mixed = c->precision == OFDFT_MIXED;
    const CgState &h = *c->st_h[0];
    stats.iterations = h.it;
    stats.evaluations = h.nevals;
    stats.gnorm = h.gnorm;
    stats.status = h.status == kCgStagnated ? OFDFT_OK : h.status;
    if (graph) c->launches += graph_launches(c, h);
    if (mixed) {
        const CgState &l = *c->st_h[1];
        stats.iterations += l.it;
        stats.evaluations_lo = l.nevals;
        stats.evaluations += l.nevals;
        if (graph) c->launches += graph_launches(c, l);
    }
    es = unpack_sums(h.ev_acc, c->fp.kind == 0);
    if (h.status == OFDFT_ENUMERIC) return fail(c, OFDFT_ENUMERIC, "non-finite energy, gradient or norm");
    fill_energy(c, es, c->last);
    c->last_valid = true;
    return stats.status == OFDFT_OK ? OFDFT_OK : (ofdft_status)stats.status;
}

// ------------------------------------------------------------ batched form
// Every instance's minimisation (for a mixed context: FP32 CG, conversion,
// FP64 CG) as an independent root branch of one graph, so a batch is one
// graph launch.  Each branch is captured on its context's private stream
// into the common graph; the loop bodies are the same captures as a single
// minimisation's, so every instance takes exactly the steps it takes alone.
ofdft_status build_batch_graph(int n, ofdft_ctx *const *ctxs, cudaGraphExec_t *out)
{
    ofdft_ctx *c0 = ctxs[0];
    cudaGraph_t G = nullptr;
    if (cudaGraphCreate(&G, 0) != cudaSuccess) return fail(c0, OFDFT_EDEVICE, "cudaGraphCreate failed");
    ofdft_status r = OFDFT_OK;
    for (int i = 0; i < n && r == OFDFT_OK; ++i) {
        ofdft_ctx *c = ctxs[i];
        cudaStream_t user = c->st;
        const long long before = c->launches;
        const bool dbg_saved = c->debug_sync;
        c->st = c->cap2;
        c->debug_sync = false;
        const bool mixed = c->precision == OFDFT_MIXED;
        cudaGraphConditionalHandle o0 = 0, o1 = 0;
        cudaGraph_t b0 = nullptr, b1 = nullptr;
        cudaGraph_t cap = G;
        cudaError_t e = cudaStreamBeginCaptureToGraph(c->cap2, G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) r = fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "batch capture");
        if (r == OFDFT_OK && mixed) {
            launch_convert<double, float>(c->g.N, (const double *)c->f[0].phi, (float *)c->f[1].phi, c->st);
            r = capture_outer<float>(c, c->f[1], G, &o1, &b1);
            if (r == OFDFT_OK)
                launch_convert<float, double>(c->g.N, (const float *)c->f[1].phi, (double *)c->f[0].phi, c->st);
        }
        if (r == OFDFT_OK) r = capture_outer<double>(c, c->f[0], G, &o0, &b0);
        if (e == cudaSuccess) {
            e = cudaStreamEndCapture(c->cap2, &cap);
            if (e != cudaSuccess && r == OFDFT_OK) r = fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "batch capture");
        }
        if (r == OFDFT_OK && mixed) r = capture_body<float>(c, c->f[1], o1, b1);
        if (r == OFDFT_OK) r = capture_body<double>(c, c->f[0], o0, b0);
        c->st = user;
        c->debug_sync = dbg_saved;
        c->launches = before;
        if (r != OFDFT_OK && c != c0) c0->err = c->err;
    }
    if (r == OFDFT_OK) {
        cudaError_t e = cudaGraphInstantiate(out, G, 0);
        if (e != cudaSuccess) {
            *out = nullptr;
            r = fail(c0, OFDFT_EDEVICE, cudaGetErrorString(e), "batch graph instantiation");
        }
    }
    cudaGraphDestroy(G);
    return r;
}

// One graph launch for the whole batch on the first context's stream, after
// the work already queued on every context's stream; the contexts' streams
// then wait for it.  The executable graph is kept by the first context and
// reused while the same contexts (same launch shapes) come in the same order.
ofdft_status batch_graph_minimize(int n, ofdft_ctx *const *ctxs, double gtol, int maxit, ofdft_energy *E,
                                  ofdft_stats *stats)
{
    ofdft_ctx *c0 = ctxs[0];
    ofdft_ctx *const c = c0;   // device errors are reported on the first context
    std::vector<unsigned long long> key;
    for (int i = 0; i < n; ++i) {
        key.push_back(ctxs[i]->uid);
        key.push_back(ctxs[i]->shape_epoch);
    }
    if (!c0->batch_exec || c0->batch_key != key) {
        if (c0->batch_exec) cudaGraphExecDestroy(c0->batch_exec);
        c0->batch_exec = nullptr;
        c0->batch_key.clear();
        ofdft_status r = build_batch_graph(n, ctxs, &c0->batch_exec);
        if (r != OFDFT_OK) return r;
        c0->batch_key = key;
    }
    cudaStream_t S = c0->st;
    for (int i = 0; i < n; ++i) {
        ofdft_ctx *ci = ctxs[i];
        if (ci != c0) {
            CK(cudaEventRecord(ci->done_ev, ci->st));
            CK(cudaStreamWaitEvent(S, ci->done_ev, 0));
        }
        if (ci->precision == OFDFT_MIXED && write_config(ci, 1, gtol, maxit, kStagnateIts, S) != OFDFT_OK)
            return OFDFT_EDEVICE;
        if (write_config(ci, 0, gtol, maxit, 0, S) != OFDFT_OK) return OFDFT_EDEVICE;
    }
    CK(cudaGraphLaunch(c0->batch_exec, S));
    for (int i = 0; i < n; ++i) {
        ofdft_ctx *ci = ctxs[i];
        for (int k = 0; k < (ci->precision == OFDFT_MIXED ? 2 : 1); ++k)
            CK(cudaMemcpyAsync(ci->st_h[k], ci->f[k].cs, sizeof(CgState), cudaMemcpyDeviceToHost, S));
    }
    CK(cudaEventRecord(c0->done_ev, S));
    for (int i = 1; i < n; ++i) CK(cudaStreamWaitEvent(ctxs[i]->st, c0->done_ev, 0));
    CK(cudaEventSynchronize(c0->done_ev));
    CK(cudaGetLastError());
    ofdft_status first = OFDFT_OK;
    for (int i = 0; i < n; ++i) {
        ofdft_stats st{};
        EvalScalars es;
        ofdft_status s = finish_minimize(ctxs[i], true, st, es);
        if (E) E[i] = s == OFDFT_OK || s == OFDFT_ENOCONV ? ctxs[i]->last : ofdft_energy{};
        if (stats) stats[i] = st;
        if (s != OFDFT_OK && first == OFDFT_OK) first = s;
    }
    return first;
}

ofdft_status run_minimize(ofdft_ctx *c, double gtol, int maxit, ofdft_stats &stats, EvalScalars &es)
{
    stats = ofdft_stats{};
    ofdft_status s = minimize_start(c, gtol, maxit);
    if (s != OFDFT_OK) return s;
    return minimize_wait(c, stats, es);
}

// ------------------------------------------------ truncated Newton
// The paper's alternative to CG (Sec. II names CG and truncated Newton and
// gives no details).  Reading, the same steps as the oracle's minimize_tn:
// each outer step solves H d = -g on the tangent space (orthogonal to phi)
// by an inner CG, truncated when ||r|| <= eta ||g||, after inner_max steps
// or at non-positive curvature (then the last iterate, or -g at the first
// step).  H p is the central difference of the gradient map
// g(psi) = 2 psi (v[psi^2] - mu) along p (mu held), projected orthogonal to
// phi; the step then takes the CG's norm-preserving rotation and line
// search from the Newton angle min(||d|| / ||phi||, 1).  Host-driven: the
// field work runs in the FP64 field set's kernels, the scalars on the host.
struct TnVec {
    double *x = nullptr, *r = nullptr, *p = nullptr, *hp = nullptr, *psi = nullptr, *gp = nullptr,
           *gq = nullptr, *vpsi = nullptr, *b = nullptr;
};

ofdft_status tn_dot(ofdft_ctx *c, const double *a, const double *b, double &out)
{
    const int nb = launch_dot<double>(c->g.N, a, b, c->part, c->st);
    launch_reduce(c->part, nb, 1, c->scal, c->st);
    c->launches += 2;
    if (sync_read(c, 1) != OFDFT_OK) return OFDFT_EDEVICE;
    out = c->scal_h[0];
    return OFDFT_OK;
}

double e_elec_host(const ofdft_ctx *c, const EvalScalars &es) { return es.EH + es.Eloc + c->g.dV * (es.FS + es.FXC); }

// One trial of the line search: phit = phi cos + dhat sin, its energy and
// dE/dtheta (the same sums the device line search reads).
ofdft_status tn_trial(ofdft_ctx *c, FieldSet &f, double th, EvalScalars &es)
{
    ofdft_status s = enqueue_eval<double>(c, f, (double *)f.phit, (const double *)f.phi, (const double *)f.dhat,
                                          cos(th), sin(th), nullptr, (double *)f.vt, false, c->scal);
    if (s != OFDFT_OK) return s;
    if (sync_read(c, 18) != OFDFT_OK) return OFDFT_EDEVICE;
    es = unpack_sums(c->scal_h, c->fp.kind == 0);
    return OFDFT_OK;
}

// The gradient map at psi = phi + h p: gout = 2 psi (v[psi^2] - mu).
ofdft_status tn_grad_at(ofdft_ctx *c, FieldSet &f, const TnVec &w, double h, double mu, double *gout)
{
    const long long N = c->g.N;
    launch_axpby<double>(N, 1.0, (const double *)f.phi, h, w.p, w.psi, c->st);
    ofdft_status s = enqueue_eval<double>(c, f, w.psi, nullptr, nullptr, 1.0, 0.0, nullptr, w.vpsi, false, c->scal);
    if (s != OFDFT_OK) return s;
    launch_cg_grad<double>(N, w.psi, w.vpsi, mu, nullptr, gout, nullptr, c->part, c->st);
    c->launches += 2;
    return OFDFT_OK;
}

ofdft_status minimize_tn(ofdft_ctx *c, double gtol, int maxit, int inner_max, double eta, ofdft_stats &stats,
                         int &nhess, EvalScalars &es)
{
    FieldSet &f = c->f[0];
    const long long N = c->g.N;
    const double dV = c->g.dV;
    const double fd_rel = 1e-4, ls_tol = 0.1, e_tol = 1e-11;
    const int max_ls = 20;
    stats = ofdft_stats{};
    nhess = 0;
    TnVec w;
    double **bufs[] = {&w.x, &w.r, &w.p, &w.hp, &w.psi, &w.gp, &w.gq, &w.vpsi, &w.b};
    for (double **b : bufs) CK(cudaMallocAsync((void **)b, N * sizeof(double), c->st));
    auto release = [&]() {
        for (double **b : bufs)
            if (*b) cudaFreeAsync(*b, c->st);
    };
    double *phi = (double *)f.phi, *v = (double *)f.v, *g = (double *)f.g, *d = (double *)f.d;
    ofdft_status s = OFDFT_OK;
    int nevals = 0, it = 0;
    double mu = 0.0, gnorm = 0.0, pp = 0.0;
    stats.status = OFDFT_ENOCONV;
#define TN_TRY(call)                \
    do {                            \
        s = (call);                 \
        if (s != OFDFT_OK) {        \
            release();              \
            return s;               \
        }                           \
    } while (0)
    // normalise (dV sum phi^2 = N_e) and evaluate
    TN_TRY(tn_dot(c, phi, phi, pp));
    if (!(pp > 0.0) || !std::isfinite(pp)) {
        release();
        return fail(c, OFDFT_ENUMERIC, "non-finite or zero density");
    }
    launch_scale<double>(N, phi, sqrt(c->Ne / (dV * pp)), nullptr, c->st);
    TN_TRY(evaluate<double>(c, f, phi, v, false, es));
    nevals = 1;
    auto grad = [&]() -> ofdft_status {
        mu = es.PHI2V / es.PHI2;
        launch_cg_grad<double>(N, phi, v, mu, nullptr, g, nullptr, c->part, c->st);
        c->launches++;
        double gg;
        ofdft_status r = tn_dot(c, g, g, gg);
        gnorm = sqrt(dV * gg);
        return r;
    };
    TN_TRY(grad());
    while (it < maxit) {
        if (!std::isfinite(gnorm)) {
            release();
            return fail(c, OFDFT_ENUMERIC, "non-finite gradient");
        }
        if (gnorm < gtol) {
            stats.status = OFDFT_OK;
            break;
        }
        TN_TRY(tn_dot(c, phi, phi, pp));
        double pg;
        TN_TRY(tn_dot(c, phi, g, pg));
        launch_axpby<double>(N, -1.0, g, pg / pp, phi, w.b, c->st);          // b = -proj(g)
        launch_fill<double>(N, w.x, 0.0, c->st);
        CK(cudaMemcpyAsync(w.r, w.b, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(w.p, w.b, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        c->launches += 2;
        double rr, bb;
        TN_TRY(tn_dot(c, w.r, w.r, rr));
        bb = rr;
        const double bn = sqrt(bb);
        for (int j = 0; j < inner_max; ++j) {
            double ppp;
            TN_TRY(tn_dot(c, w.p, w.p, ppp));
            const double h = fd_rel * sqrt(pp / ppp);
            TN_TRY(tn_grad_at(c, f, w, h, mu, w.gp));
            TN_TRY(tn_grad_at(c, f, w, -h, mu, w.gq));
            nevals += 2;
            ++nhess;
            launch_axpby<double>(N, 0.5 / h, w.gp, -0.5 / h, w.gq, w.hp, c->st);
            c->launches++;
            double ph;
            TN_TRY(tn_dot(c, phi, w.hp, ph));
            launch_axpby<double>(N, 1.0, w.hp, -ph / pp, phi, w.hp, c->st);   // project
            c->launches++;
            double pHp;
            TN_TRY(tn_dot(c, w.p, w.hp, pHp));
            if (!(pHp > 0.0)) {
                if (j == 0) CK(cudaMemcpyAsync(w.x, w.b, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
                break;
            }
            const double a = rr / pHp;
            launch_axpby<double>(N, 1.0, w.x, a, w.p, w.x, c->st);
            launch_axpby<double>(N, 1.0, w.r, -a, w.hp, w.r, c->st);
            c->launches += 2;
            double rr_new;
            TN_TRY(tn_dot(c, w.r, w.r, rr_new));
            if (sqrt(rr_new) <= eta * bn) break;
            launch_axpby<double>(N, 1.0, w.r, rr_new / rr, w.p, w.p, c->st);
            c->launches++;
            rr = rr_new;
        }
        // d = proj(x), or -proj(g) when it does not descend
        double px;
        TN_TRY(tn_dot(c, phi, w.x, px));
        launch_axpby<double>(N, 1.0, w.x, -px / pp, phi, d, c->st);
        c->launches++;
        double dg;
        TN_TRY(tn_dot(c, d, g, dg));
        if (dg >= 0.0) CK(cudaMemcpyAsync(d, w.b, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        double dd;
        TN_TRY(tn_dot(c, d, d, dd));
        const double theta1 = std::min(sqrt(dd / pp), 1.0);
        // dhat = d sqrt(pp/dd) and D0 = dV sum 2 phi v dhat (the CG's kernel with c1 = 0)
        const int nb = launch_cg_dhat<double>(N, g, d, phi, v, 0.0, sqrt(pp / dd), 0, nullptr, (double *)f.dhat,
                                              c->part, c->st);
        launch_reduce(c->part, nb, 1, c->scal, c->st);
        c->launches += 2;
        if (sync_read(c, 1) != OFDFT_OK) {
            release();
            return OFDFT_EDEVICE;
        }
        const double D0 = dV * c->scal_h[0];
        // line search on theta (the CG's rules)
        const double E0 = e_elec_host(c, es);
        double lo = 0.0, Dlo = D0, hi = -1.0, Dhi = 0.0, pa = 0.0, Da = D0, th = theta1;
        bool hi_nod = false, accepted = false;
        EvalScalars et;
        for (int k = 0; k < max_ls && !accepted; ++k) {
            TN_TRY(tn_trial(c, f, th, et));
            ++nevals;
            const double D = dV * et.DTH;
            const bool up = e_elec_host(c, et) > E0 + 1e-4 * th * D0 + e_tol * fabs(E0);
            if (!up && fabs(D) <= ls_tol * fabs(D0)) {
                accepted = true;
                break;
            }
            if (up) {
                hi = th;
                Dhi = D;
                hi_nod = !(D > 0.0);
            } else if (D < 0.0) {
                lo = th;
                Dlo = D;
            } else {
                hi = th;
                Dhi = D;
                hi_nod = false;
            }
            double nxt;
            if (hi < 0.0) {
                nxt = 4.0 * th;
                if (D > Da) nxt = std::min(th - D * (th - pa) / (D - Da), 4.0 * th);
                nxt = std::max(nxt, 1.1 * th);
                pa = th;
                Da = D;
            } else if (hi_nod) {
                nxt = 0.5 * (lo + hi);
            } else {
                nxt = lo - Dlo * (hi - lo) / (Dhi - Dlo);
                const double wdt = hi - lo;
                nxt = std::min(std::max(nxt, lo + 0.01 * wdt), hi - 0.01 * wdt);
            }
            th = std::min(nxt, 1.5);
        }
        if (!accepted && lo > 0.0) {   // the best descent point found
            TN_TRY(tn_trial(c, f, lo, et));
            ++nevals;
            accepted = true;
        }
        if (!accepted) {
            stats.status = OFDFT_ENOCONV;
            break;
        }
        CK(cudaMemcpyAsync(phi, f.phit, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(v, f.vt, N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        es = et;
        ++it;
        TN_TRY(grad());
    }
#undef TN_TRY
    release();
    stats.iterations = it;
    stats.evaluations = nevals;
    stats.gnorm = gnorm;
    fill_energy(c, es, c->last);
    c->last_valid = true;
    return (ofdft_status)stats.status;
}

ofdft_status forces_now(ofdft_ctx *c, EvalScalars &es)
{
    FieldSet &f = c->f[0];
    ofdft_status s = evaluate<double>(c, f, (double *)f.phi, (double *)f.vt, true, es);
    if (s != OFDFT_OK) return s;
    const GridInfo &g = c->g;
    const double2 *nG = (const double2 *)f.spec + f.spec_stride;
    const PhaseTablesDD *dd = g.dd ? &c->pdd : nullptr;
    size_t need = (size_t)c->nat * lpp_force_chunks(g, c->nat, dd != nullptr) * 3 + 16;
    if (need > c->fpart_len) {
        if (c->fpart) cudaFreeAsync(c->fpart, c->st);
        c->fpart = nullptr;
        CK(cudaMallocAsync((void **)&c->fpart, need * sizeof(double), c->st));
        c->fpart_len = need;
    }
    // the third spectrum is free after an evaluation (ftTF and GGA alike)
    double2 *cn = (double2 *)f.spec + 2 * f.spec_stride;
    int nchunk = launch_lpp_forces<double>(g, c->nat, c->Zd, c->px, c->py, c->pz, dd, nG, cn, c->fpart, c->st);
    launch_force_reduce(c->nat, nchunk, c->fpart, c->Fd, 0, c->st);
    c->launches += 3;
    std::vector<double> F(3 * c->nat), Fe(3 * c->nat);
    CK(cudaMemcpyAsync(F.data(), c->Fd, F.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(Fe.data(), c->ewF, Fe.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (size_t i = 0; i < F.size(); ++i) F[i] += Fe[i];
    CK(cudaMemcpyAsync(c->Fd, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    return OFDFT_OK;
}

void free_fieldset(FieldSet &f, cudaStream_t st)
{
    void *ptrs[] = {f.phi, f.phit, f.dhat, f.g, f.gprev, f.d, f.v, f.vt, f.vpart, f.spec, f.vext, f.tab,
                    f.tw[0], f.tw[1], f.tw[2], f.cs};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, st);
    if (f.graph) cudaGraphExecDestroy(f.graph);
    f = FieldSet{};
}

// Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// context's stream), so creating and destroying contexts never waits for
// the work of other contexts on the device.
void free_ctx(ofdft_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->st) cudaStreamSynchronize(c->st);
    free_fieldset(c->f[0], c->st);
    free_fieldset(c->f[1], c->st);
    void *ptrs[] = {c->phiprev, c->part, c->scal, c->Rd, c->Zd, c->Fd, c->Vd, c->Md, c->nh, c->px, c->py,
                    c->pz, c->pdd.xT, c->fpart, c->Gv, c->wG, c->eion, c->ewF, c->ewpart, c->Se};
    for (void *p : ptrs)
        if (p) cudaFreeAsync(p, c->st);
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->scal_h) cudaFreeHost(c->scal_h);
    for (int k = 0; k < 2; ++k) {
        if (c->cfg_h[k]) cudaFreeHost(c->cfg_h[k]);
        if (c->st_h[k]) cudaFreeHost(c->st_h[k]);
    }
    if (c->batch_exec) cudaGraphExecDestroy(c->batch_exec);
    if (c->done_ev) cudaEventDestroy(c->done_ev);
    for (cudaEvent_t e : c->tev) cudaEventDestroy(e);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    if (c->cap2) cudaStreamDestroy(c->cap2);
    for (cudaStream_t a : c->aux)
        if (a) cudaStreamDestroy(a);
    for (cudaEvent_t e : c->fj)
        if (e) cudaEventDestroy(e);
    delete c;
}

template <typename T> ofdft_status alloc_fieldset(ofdft_ctx *c, FieldSet &f)
{
    const GridInfo &g = c->g;
    size_t rb = (size_t)g.N * sizeof(T);
    size_t cb = ((size_t)g.NH * sizeof(cplx<T>) + 255) & ~(size_t)255;
    void **fields[] = {&f.phi, &f.phit, &f.dhat, &f.g, &f.gprev, &f.d, &f.v, &f.vt, &f.vpart};
    for (void **p : fields) CK(cudaMallocAsync(p, rb, c->st));
    CK(cudaMallocAsync((void **)&f.spec, 4 * cb, c->st));
    f.spec_stride = cb / sizeof(cplx<T>);
    // v_ext(G); the Heine-Abarenkov form and triclinic cells append the pressure weights
    CK(cudaMallocAsync((void **)&f.vext, (size_t)((g.lpp || g.tri) ? 2 : 1) * g.NH * sizeof(cplx<T>), c->st));
    // temperature table; FP64 sets append its double-float split (hi, lo
    // binary32 pairs) and the double-float VT84F enhancement table for the
    // double-float pointwise functional
    const std::vector<double> &tab = tfunc_table_host();
    std::vector<T> tt(tab.begin(), tab.end());
    if (sizeof(T) == 8) {
        std::vector<double> dd((size_t)kDdTabSize);
        dd_tables_fill(tab.data(), dd.data());
        tt.assign(dd.begin(), dd.end());
    }
    CK(cudaMallocAsync((void **)&f.tab, tt.size() * sizeof(T), c->st));
    CK(cudaMemcpyAsync(f.tab, tt.data(), tt.size() * sizeof(T), cudaMemcpyHostToDevice, c->st));
    int n3[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a)
        if (upload_twiddles<T>(c, f, a, n3[a]) != OFDFT_OK) return OFDFT_EDEVICE;
    CK(cudaMallocAsync((void **)&f.cs, sizeof(CgState), c->st));
    f.gt = c->g;
    CK(cudaMemsetAsync(f.cs, 0, sizeof(CgState), c->st));
    f.valid = true;
    return OFDFT_OK;
}

ofdft_status alloc_ctx(ofdft_ctx *c)
{
    const GridInfo &g = c->g;
    if (alloc_fieldset<double>(c, c->f[0]) != OFDFT_OK) return OFDFT_ENOMEM;
    if (c->precision == OFDFT_MIXED && alloc_fieldset<float>(c, c->f[1]) != OFDFT_OK) return OFDFT_ENOMEM;
    CK(cudaMallocAsync((void **)&c->phiprev, (size_t)g.N * sizeof(double), c->st));
    const int ntk = (g.K + 3) / 4;              // narrowest column tile the autotuner tries
    size_t need = (size_t)3 * g.ny * ntk + (size_t)15 * ((size_t)g.nx * g.ny / 2) + 64;
    need = std::max<size_t>(need, 5 * 1216 + 64);
    CK(cudaMallocAsync((void **)&c->part, need * sizeof(double), c->st));
    c->part_len = need;
    CK(cudaMallocAsync((void **)&c->scal, 64 * sizeof(double), c->st));
    CK(cudaMallocHost(&c->scal_h, 64 * sizeof(double)));
    for (int k = 0; k < 2; ++k) {
        CK(cudaMallocHost(&c->cfg_h[k], sizeof(CgState)));
        CK(cudaMallocHost(&c->st_h[k], sizeof(CgState)));
        memset(c->st_h[k], 0, sizeof(CgState));
    }
    CK(cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming));
    const int nat = c->nat;
    CK(cudaMallocAsync((void **)&c->Rd, 3 * nat * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->Zd, nat * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->Fd, 3 * nat * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->Vd, 3 * nat * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->Md, nat * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->nh, 4 * sizeof(double), c->st));
    CK(cudaMallocAsync((void **)&c->px, (size_t)nat * g.nx * sizeof(double2), c->st));
    CK(cudaMallocAsync((void **)&c->py, (size_t)nat * g.ny * sizeof(double2), c->st));
    CK(cudaMallocAsync((void **)&c->pz, (size_t)nat * g.K * sizeof(double2), c->st));
    if (g.dd) {
        const size_t nx = (size_t)nat * g.nx, ny = (size_t)nat * g.ny, nk = (size_t)nat * g.K;
        CK(cudaMallocAsync((void **)&c->pdd.xT, (nx + ny + 2 * nk) * sizeof(double2), c->st));
        c->pdd.yT = c->pdd.xT + nx;
        c->pdd.zT = c->pdd.yT + ny;
        c->pdd.zd = c->pdd.zT + nk;
    }
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
    // leave room for the kernels' static shared memory (block reductions)
    size_t dyn = (size_t)optin - 8192;
    if (field_smem_max(g, sizeof(double2)) > dyn)
        return fail(c, OFDFT_EINVAL, "grid too large for the shared-memory tiles");
    CK(set_field_smem_limits<double>(dyn));
    CK(set_field_smem_limits<float>(dyn));
    CK(cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking));
    for (cudaStream_t &a : c->aux) CK(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    for (cudaEvent_t &e : c->fj) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return OFDFT_OK;
}

ofdft_status normalize_phi64(ofdft_ctx *c)
{
    FieldSet &f = c->f[0];
    int nb = launch_sumsq<double>(c->g.N, (const double *)f.phi, c->part, c->st);
    launch_reduce(c->part, nb, 1, c->scal, c->st);
    c->launches += 2;
    if (sync_read(c, 1) != OFDFT_OK) return OFDFT_EDEVICE;
    double ss = c->scal_h[0] * c->g.dV;
    if (!(ss > 0.0) || !isfinite(ss)) return fail(c, OFDFT_ENUMERIC, "phi has zero or non-finite norm");
    launch_scale<double>(c->g.N, (double *)f.phi, sqrt(c->Ne / ss), nullptr, c->st);
    c->launches++;
    return OFDFT_OK;
}

// Device bytes of one context (upper estimate mirroring alloc_ctx and
// setup_ewald; the Ewald G count is bounded by its cube, which depends on
// nat only for the splitting used there).
double footprint_bytes(const int grid[3], int nat, int precision)
{
    const double nx = grid[0], ny = grid[1], nz = grid[2];
    const double K = std::floor(nz / 2) + 1, N = nx * ny * nz, NH = nx * ny * K;
    const double tab = (double)tfunc_table_host().size();
    auto fieldset = [&](double sz) {
        double cb = std::ceil(NH * 2 * sz / 256.0) * 256.0;
        // v_ext(G) counted twice: the Heine-Abarenkov form adds its pressure weights
        return 9 * N * sz + 4 * cb + 2 * NH * 2 * sz + tab * sz + (nx + ny + nz) * 2 * sz + sizeof(CgState);
    };
    double b = fieldset(8.0) + (precision == OFDFT_MIXED ? fieldset(4.0) : 0.0);
    b += N * 8;                                                        // phiprev
    b += (3 * ny * std::ceil(K / 4) + 15 * (nx * ny / 2) + 64) * 8 + 64 * 8;  // partials, scalars
    b += nat * 11.0 * 8 + 32 + nat * (2 * nx + 2 * ny + 3 * K) * 16.0;  // ions, phase factors (+ double-float)
    b += nat * std::max(1216.0, (double)lpp_force_chunks_dd((long long)(nx * ny), nat)) * 3 * 8 + 16 * 8;   // force partials
    double km = std::ceil(4.27 * std::pow((double)nat, 1.0 / 6.0)) + 1;
    b += std::pow(2 * km + 1, 3) * 6 * 8 + nat * 4.0 * 8;             // Ewald tables
    return 1.05 * b + 8.0 * (1 << 20);                                 // pool granularity, graphs
}

ofdft_status busy(ofdft_ctx *c)
{
    return c->pending ? fail(c, OFDFT_EBUSY, "a minimisation is in flight (call ofdft_minimize_wait)") : OFDFT_OK;
}

#define NOT_BUSY(c)                              \
    do {                                         \
        if (busy(c) != OFDFT_OK) return OFDFT_EBUSY; \
    } while (0)

// ------------------------------------------------------------ autotuner
struct TuneKey {
    int nx, ny, nz, prec;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(nx, ny, nz, prec) < std::tie(o.nx, o.ny, o.nz, o.prec);
    }
};
std::mutex g_tune_mu;
struct Tuned {
    int zP, tk, zth, xth;
    int mp[3];   // largest power-of-two radix per axis
    int dk, dth; // derivative passes: tile width, threads
    int dws;     // derivative passes with warp-owned lines
};

// Rebuild axis a's Stockham schedule with power-of-two radices up to m (the
// twiddle tables do not depend on the schedule).
void set_radix(FieldSet &f, int a, int m)
{
    const void *twf = f.ax[a].twf;
    f.ax[a] = fft_axis(f.ax[a].n, f.ax[a].tw, m);
    f.ax[a].twf = twf;
}
std::map<TuneKey, Tuned> g_tune;

// Mean time of `reps` evaluations of field set f at its current phi.
template <typename T> ofdft_status time_evals(ofdft_ctx *c, FieldSet &f, int reps, float &ms)
{
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    ofdft_status r = enqueue_eval<T>(c, f, (T *)f.phi, nullptr, nullptr, 1.0, 0.0, nullptr, (T *)f.vt, false, c->scal);
    cudaEventRecord(e0, c->st);
    for (int i = 0; i < reps && r == OFDFT_OK; ++i)
        r = enqueue_eval<T>(c, f, (T *)f.phi, nullptr, nullptr, 1.0, 0.0, nullptr, (T *)f.vt, false, c->scal);
    cudaEventRecord(e1, c->st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != OFDFT_OK) return r;
    if (e != cudaSuccess) return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "autotune timing");
    ms /= (float)reps;
    return OFDFT_OK;
}

// Pick the launch shapes by timing whole evaluations: tile width and
// threads of the y/x passes together, then line pairs per block and threads
// of the z passes, then tile width and threads of the derivative passes,
// then each axis's radix schedule.
template <typename T> ofdft_status autotune_set(ofdft_ctx *c, int k, int reps)
{
    FieldSet &f = c->f[k];
    const TuneKey key{c->g.nx, c->g.ny, c->g.nz, (int)sizeof(T)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            f.gt.zP = it->second.zP;
            f.gt.tk = it->second.tk;
            f.gt.zth = it->second.zth;
            f.gt.xth = it->second.xth;
            f.gt.dk = it->second.dk;
            f.gt.dth = it->second.dth;
            f.gt.dws = it->second.dws;
            for (int a = 0; a < 3; ++a) set_radix(f, a, it->second.mp[a]);
            if (f.graph) cudaGraphExecDestroy(f.graph);
            f.graph = nullptr;
            c->shape_epoch++;
            return OFDFT_OK;
        }
    }
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
    const size_t dyn = (size_t)optin - 8192;
    GridInfo best = f.gt;
    float best_ms = 1e30f;
    // try g (if it fits); keep it when faster than the best so far
    auto trial = [&](const GridInfo &g) -> ofdft_status {
        if (field_smem_max(g, sizeof(cplx<T>)) > dyn) return OFDFT_OK;
        f.gt = g;
        float ms;
        ofdft_status r = time_evals<T>(c, f, reps, ms);
        if (r == OFDFT_OK && ms < best_ms) {
            best_ms = ms;
            best = g;
        }
        return r;
    };
    const int tmax = fft_max_threads();
    // the y/x passes: tile width and threads together (a stage's butterflies
    // per tile set how many threads can work)
    {
        const GridInfo base = best;
        for (int tk : {4, 8, 16})
            for (int th : {128, 256, 512}) {
                if ((tk > base.K && tk != 4) || th > tmax) continue;
                GridInfo g = base;
                g.tk = tk;
                g.xth = th;
                ofdft_status r = trial(g);
                if (r != OFDFT_OK) return r;
            }
    }
    // the z passes: line pairs per block and threads together (the FP64 z
    // passes keep at most 256 threads)
    {
        const GridInfo base = best;
        for (int zp : {1, 2, 4, 8})
            for (int th : {128, 256, 512}) {
                if ((long long)zp * base.nz > 2048 || (long long)zp > (long long)base.nx * base.ny / 2) continue;
                if (th > tmax || (sizeof(T) == 8 && th > 256)) continue;
                GridInfo g = base;
                g.zP = zp;
                g.zth = th;
                ofdft_status r = trial(g);
                if (r != OFDFT_OK) return r;
            }
    }
    // the derivative passes' tile width and threads together (GGA only)
    if (c->fp.kind != 0) {
        const GridInfo base = best;
        for (int dk : {4, 8, 16})
            for (int th : {64, 128, 256}) {
                if (th > tmax) continue;
                GridInfo g = base;
                g.dk = dk;
                g.dth = th;
                g.dws = 0;
                ofdft_status r = trial(g);
                if (r != OFDFT_OK) return r;
            }
        // warp-owned lines: 1, 2 or 4 lines a warp
        for (int dk : {8, 16})
            for (int lpw : {1, 2, 4}) {
                const int th = 32 * dk / lpw;
                if (th > tmax || th < 64) continue;
                GridInfo g = base;
                g.dk = dk;
                g.dth = th;
                g.dws = 1;
                ofdft_status r = trial(g);
                if (r != OFDFT_OK) return r;
            }
    }
    f.gt = best;
    // the Stockham schedule of each axis: power-of-two radices up to 8 or
    // up to 4 (fewer stages against shorter butterflies; same twiddles)
    int mp[3];
    for (int a = 0; a < 3; ++a) {
        best_ms = 1e30f;
        mp[a] = f.ax[a].mp;
        for (int m : {4, 8}) {
            set_radix(f, a, m);
            float ms;
            ofdft_status r = time_evals<T>(c, f, reps, ms);
            if (r != OFDFT_OK) return r;
            if (ms < best_ms) {
                best_ms = ms;
                mp[a] = m;
            }
        }
        set_radix(f, a, mp[a]);
    }
    if (f.graph) cudaGraphExecDestroy(f.graph);
    f.graph = nullptr;
    c->shape_epoch++;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = Tuned{best.zP, best.tk, best.zth, best.xth, {mp[0], mp[1], mp[2]}, best.dk, best.dth, best.dws};
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
    p->pointwise = OFDFT_PW_F32X2;
    p->lpp = OFDFT_LPP_GAUSS;
    p->lpp_A = 6.18;      // Eq. (E4A), hydrogen
    p->lpp_qc = 29.97;
}

ofdft_status ofdft_setup(const double cell[9], const int grid[3], int nat, const double *ions,
                         const double *Z, double T_kelvin, int functional, const ofdft_params *params,
                         ofdft_ctx **out)
{
    if (!out) return fail(nullptr, OFDFT_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cell || !grid || !ions || !Z || nat <= 0) return fail(nullptr, OFDFT_EINVAL, "NULL input or nat <= 0");
    bool tri = false;
    for (int i = 0; i < 9; ++i) {
        if (!isfinite(cell[i])) return fail(nullptr, OFDFT_EINVAL, "non-finite cell");
        if (i % 4 != 0 && cell[i] != 0.0) tri = true;
    }
    const double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) -
                       cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
                       cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
    if (!tri && !(cell[0] > 0 && cell[4] > 0 && cell[8] > 0))
        return fail(nullptr, OFDFT_EINVAL, "non-positive cell edge");
    if (tri && !(det > 0.0)) return fail(nullptr, OFDFT_EINVAL, "cell vectors must be right-handed (det > 0)");
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
    if (p.pointwise != OFDFT_PW_F32X2 && p.pointwise != OFDFT_PW_F64)
        return fail(nullptr, OFDFT_EINVAL, "bad pointwise arithmetic");
    const bool dd = p.pointwise == OFDFT_PW_F32X2;
    if (p.lpp != OFDFT_LPP_GAUSS && p.lpp != OFDFT_LPP_HA) return fail(nullptr, OFDFT_EINVAL, "unknown lpp");
    if (p.lpp == OFDFT_LPP_HA) {
        if (!isfinite(p.lpp_A) || !(p.lpp_qc > 0.0) || !isfinite(p.lpp_qc))
            return fail(nullptr, OFDFT_EINVAL, "Heine-Abarenkov LPP needs finite A and qc > 0");
        for (int i = 1; i < nat; ++i)
            if (Z[i] != Z[0])
                return fail(nullptr, OFDFT_EINVAL, "Heine-Abarenkov LPP takes one species (equal Z)");
    }
    for (int i = 0; i < nat; ++i) {
        if (!(Z[i] > 0.0)) return fail(nullptr, OFDFT_EINVAL, "Z must be > 0");
        for (int a = 0; a < 3; ++a)
            if (!isfinite(ions[3 * i + a])) return fail(nullptr, OFDFT_EINVAL, "non-finite ion position");
    }
    ofdft_ctx *c = new (std::nothrow) ofdft_ctx();
    if (!c) return fail(nullptr, OFDFT_ENOMEM, "host allocation failed");
    static std::atomic<unsigned long long> next_uid{1};
    c->uid = next_uid++;
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
    g.tri = tri ? 1 : 0;
    if (tri) {
        for (int k = 0; k < 9; ++k) g.Am[k] = cell[k];
        g.Lx = sqrt(cell[0] * cell[0] + cell[1] * cell[1] + cell[2] * cell[2]);
        g.Ly = sqrt(cell[3] * cell[3] + cell[4] * cell[4] + cell[5] * cell[5]);
        g.Lz = sqrt(cell[6] * cell[6] + cell[7] * cell[7] + cell[8] * cell[8]);
        g.omega = det;
    } else {
        g.Lx = cell[0];
        g.Ly = cell[4];
        g.Lz = cell[8];
        g.omega = g.Lx * g.Ly * g.Lz;
    }
    g.dV = g.omega / (double)g.N;
    g.rc = p.rc;
    g.lpp = p.lpp;
    g.ha_A = p.lpp_A;
    g.ha_qc = p.lpp_qc;
    g.ha_Z = Z[0];
    grid_reciprocal(g);
    g.dd = dd ? 1 : 0;
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
    const char *dbgenv = getenv("OFDFT_DEBUG_SYNC");
    c->debug_sync = dbgenv && dbgenv[0] == '1';
    const char *gr = getenv("OFDFT_NO_GRAPHS");
    c->use_graphs = !(gr && gr[0] == '1');
    // OFDFT_DLINE_WS="dk,threads": start from derivative passes with
    // warp-owned lines (checks of that kernel form; ofdft_autotune may
    // choose it by itself)
    const char *ws = getenv("OFDFT_DLINE_WS");
    if (ws) {
        int dk = 0, th = 0;
        if (sscanf(ws, "%d,%d", &dk, &th) == 2 && (dk == 8 || dk == 16) && th >= 32 && th <= 256 && th % 32 == 0 &&
            dk % (th / 32) == 0) {
            c->g.dws = 1;
            c->g.dk = dk;
            c->g.dth = th;
        }
    }
    ofdft_status s = alloc_ctx(c);
    if (s == OFDFT_OK) s = setup_ewald(c);
    if (s != OFDFT_OK) {
        g_setup_error = c->err;
        free_ctx(c);
        return s == OFDFT_EDEVICE ? OFDFT_ENOMEM : s;
    }
    cudaMemcpyAsync(c->Rd, c->R.data(), 3 * nat * sizeof(double), cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->Zd, c->Z.data(), nat * sizeof(double), cudaMemcpyHostToDevice, c->st);
    cudaMemcpyAsync(c->Md, c->masses.data(), nat * sizeof(double), cudaMemcpyHostToDevice, c->st);
    cudaMemsetAsync(c->Vd, 0, 3 * nat * sizeof(double), c->st);
    cudaMemsetAsync(c->nh, 0, 4 * sizeof(double), c->st);
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
    NOT_BUSY(c);
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
    NOT_BUSY(c);
    cudaSetDevice(c->dev);
    const long long N = c->g.N;
    FieldSet &f = c->f[0];
    if (phi) {
        CK(cudaMemcpyAsync(f.phi, phi, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
    } else {
        launch_fill<double>(N, (double *)f.phi, sqrt(c->Ne / c->g.omega), c->st);
        c->launches++;
    }
    c->last_valid = false;
    c->md_ready = false;
    return normalize_phi64(c);
}

ofdft_status ofdft_energy_potential(ofdft_ctx *c, const double *phi, ofdft_energy *E, double *v)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    NOT_BUSY(c);
    cudaSetDevice(c->dev);
    const long long N = c->g.N;
    FieldSet &f = c->f[0];
    double *ph = (double *)f.phi;
    if (phi) {
        CK(cudaMemcpyAsync(f.phit, phi, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
        ph = (double *)f.phit;
    }
    EvalScalars es;
    ofdft_status s = evaluate<double>(c, f, ph, (double *)f.vt, false, es);
    if (s != OFDFT_OK) return s;
    ofdft_energy e;
    fill_energy(c, es, e);
    if (v) {
        CK(cudaMemcpyAsync(v, f.vt, N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    if (E) *E = e;
    return OFDFT_OK;
}

ofdft_status ofdft_minimize(ofdft_ctx *c, double gtol, int maxit, ofdft_energy *E, ofdft_stats *stats)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    NOT_BUSY(c);
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

ofdft_status ofdft_minimize_tn(ofdft_ctx *c, double gtol, int maxit, int inner_max, double eta, ofdft_energy *E,
                               ofdft_stats *stats, int *hessian_products)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    NOT_BUSY(c);
    if (!(gtol > 0.0) || maxit <= 0 || inner_max <= 0 || !(eta > 0.0) || !(eta < 1.0))
        return fail(c, OFDFT_EINVAL, "gtol > 0, maxit > 0, inner_max > 0 and 0 < eta < 1 required");
    cudaSetDevice(c->dev);
    ofdft_stats st{};
    int nh = 0;
    EvalScalars es;
    ofdft_status s = minimize_tn(c, gtol, maxit, inner_max, eta, st, nh, es);
    if (stats) *stats = st;
    if (hessian_products) *hessian_products = nh;
    if (s != OFDFT_OK && s != OFDFT_ENOCONV) return s;
    if (E) *E = c->last;
    if (s == OFDFT_ENOCONV) return fail(c, OFDFT_ENOCONV, "truncated Newton did not reach the tolerance");
    return OFDFT_OK;
}

ofdft_status ofdft_minimize_start(ofdft_ctx *c, double gtol, int maxit)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    if (!(gtol > 0.0) || maxit <= 0) return fail(c, OFDFT_EINVAL, "gtol must be > 0 and maxit > 0");
    cudaSetDevice(c->dev);
    return minimize_start(c, gtol, maxit);
}

ofdft_status ofdft_minimize_query(ofdft_ctx *c)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    if (!c->pending) return OFDFT_OK;
    cudaSetDevice(c->dev);
    cudaError_t e = cudaEventQuery(c->done_ev);
    if (e == cudaErrorNotReady) return OFDFT_EBUSY;
    if (e != cudaSuccess) return fail(c, OFDFT_EDEVICE, cudaGetErrorString(e), "ofdft_minimize_query");
    return OFDFT_OK;
}

ofdft_status ofdft_minimize_wait(ofdft_ctx *c, ofdft_energy *E, ofdft_stats *stats)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    cudaSetDevice(c->dev);
    ofdft_stats st{};
    EvalScalars es;
    ofdft_status s = minimize_wait(c, st, es);
    if (stats) *stats = st;
    if (s != OFDFT_OK && s != OFDFT_ENOCONV) return s;
    if (E) *E = c->last;
    if (s == OFDFT_ENOCONV) return fail(c, OFDFT_ENOCONV, "CG did not reach the tolerance");
    return OFDFT_OK;
}

ofdft_status ofdft_batch_minimize(int n, ofdft_ctx *const *ctxs, double gtol, int maxit, ofdft_energy *E,
                                  ofdft_stats *stats)
{
    if (n < 0 || (n > 0 && !ctxs)) return fail(nullptr, OFDFT_EINVAL, "bad batch");
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]) return fail(nullptr, OFDFT_EINVAL, "NULL context in batch");
    if (!(gtol > 0.0) || maxit <= 0) return fail(nullptr, OFDFT_EINVAL, "gtol must be > 0 and maxit > 0");
    // one graph launch for the batch when every context can take part
    bool one = n > 0;
    for (int i = 0; i < n && one; ++i) {
        ofdft_ctx *c = ctxs[i];
        one = graphs_on(c) && !c->pending && c->dev == ctxs[0]->dev;
        for (int j = 0; j < i && one; ++j) one = ctxs[j] != c;
    }
    if (one) {
        cudaSetDevice(ctxs[0]->dev);
        return batch_graph_minimize(n, ctxs, gtol, maxit, E, stats);
    }
    ofdft_status first = OFDFT_OK;
    std::vector<char> started(n, 0);
    for (int i = 0; i < n; ++i) {
        ofdft_status s = ofdft_minimize_start(ctxs[i], gtol, maxit);
        started[i] = s == OFDFT_OK;
        if (s != OFDFT_OK && first == OFDFT_OK) first = s;
    }
    for (int i = 0; i < n; ++i) {
        ofdft_energy e{};
        ofdft_stats st{};
        ofdft_status s = started[i] ? ofdft_minimize_wait(ctxs[i], &e, &st) : OFDFT_EINVAL;
        if (!started[i]) st.status = s;
        if (E) E[i] = e;
        if (stats) stats[i] = st;
        if (s != OFDFT_OK && first == OFDFT_OK) first = s;
    }
    return first;
}

ofdft_status ofdft_footprint(const int grid[3], int nat, int precision, double *bytes)
{
    if (!grid || !bytes || nat <= 0) return fail(nullptr, OFDFT_EINVAL, "bad footprint arguments");
    for (int a = 0; a < 3; ++a)
        if (!smooth_even(grid[a])) return fail(nullptr, OFDFT_EINVAL, "bad grid");
    *bytes = footprint_bytes(grid, nat, precision);
    return OFDFT_OK;
}

ofdft_status ofdft_autotune(ofdft_ctx *c, int reps)
{
    if (!c || reps < 1) return fail(c, OFDFT_EINVAL, "NULL context or reps < 1");
    NOT_BUSY(c);
    cudaSetDevice(c->dev);
    ofdft_status s = autotune_set<double>(c, 0, reps);
    if (s == OFDFT_OK && c->f[1].valid) {
        launch_convert<double, float>(c->g.N, (const double *)c->f[0].phi, (float *)c->f[1].phi, c->st);
        s = autotune_set<float>(c, 1, reps);
    }
    return s;
}

ofdft_status ofdft_forces(ofdft_ctx *c, double *F, double *pressure)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    NOT_BUSY(c);
    cudaSetDevice(c->dev);
    EvalScalars es;
    ofdft_status s = forces_now(c, es);
    if (s != OFDFT_OK) return s;
    ofdft_energy e;
    fill_energy(c, es, e);
    if (F) {
        CK(cudaMemcpyAsync(F, c->Fd, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    if (pressure) *pressure = e.P;
    return OFDFT_OK;
}

ofdft_status ofdft_stress(ofdft_ctx *c, double *sigma, double *terms)
{
    if (!c || !sigma) return fail(c, OFDFT_EINVAL, "NULL argument");
    NOT_BUSY(c);
    cudaSetDevice(c->dev);
    FieldSet &f = c->f[0];
    const GridInfo &g = c->g;
    cudaStream_t st = c->st;
    const bool fttf = c->fp.kind == 0;
    const long long npairs = (long long)g.nx * g.ny / 2;
    const size_t nxy = (size_t)g.nx * g.ny;
    const int nbr = std::max(1, (c->nGe + 255) / 256);
    const size_t nzp = fttf ? 0 : 12 * (size_t)npairs;
    const size_t ntot = nzp + 12 * nxy + 6 * (size_t)c->nat + 7 * (size_t)nbr + 32;
    double *buf = nullptr;
    CK(cudaMallocAsync((void **)&buf, ntot * sizeof(double), st));
    double *zpart = buf, *gpart = buf + nzp, *rpart = gpart + 12 * nxy, *kpart = rpart + 6 * (size_t)c->nat;
    double *out = kpart + 7 * (size_t)nbr;
    int nbg = 0;
    ofdft_status s = enqueue_eval<double>(c, f, (double *)f.phi, nullptr, nullptr, 1.0, 0.0, nullptr,
                                          (double *)f.vt, true, c->scal, fttf ? nullptr : zpart, &nbg);
    if (s != OFDFT_OK) {
        cudaFreeAsync(buf, st);
        return s;
    }
    // out[0..5] sum W_a d_b n, [6..11] Hartree, [12..17] LPP, [18..23] Ewald real, [24..30] Ewald G
    if (!fttf) launch_reduce(zpart + 6 * (size_t)nbg, nbg, 6, out, st);
    else CK(cudaMemsetAsync(out, 0, 6 * sizeof(double), st));
    const double2 *nG = (const double2 *)f.spec + f.spec_stride;
    const int ng = launch_gstress(g, c->nat, c->Zd, c->px, c->py, c->pz, g.dd ? &c->pdd : nullptr, nG, gpart, st);
    launch_reduce(gpart, ng, 12, out + 6, st);
    const int nb = launch_ewald_stress(c->nat, c->Rd, c->Zd, ew_cell(g), c->ew_alpha, c->ew_rcut, c->ew_nimg, c->nGe,
                                       c->Gv, c->wG, (const double2 *)c->Se, rpart, kpart, st);
    launch_reduce(rpart, c->nat, 6, out + 18, st);
    launch_reduce(kpart, nb, 7, out + 24, st);
    c->launches += (fttf ? 0 : 1) + 2 + 4;
    double o[31], h[18];
    CK(cudaMemcpyAsync(o, out, sizeof(o), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h, c->scal, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(buf, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    const EvalScalars es = unpack_sums(h, fttf);
    const double V = g.omega, dV = g.dV;
    double zs = 0.0;
    for (int i = 0; i < c->nat; ++i) zs += c->Z[i];
    const double Ebg = -kPi * zs * zs / (2.0 * V * c->ew_alpha * c->ew_alpha);
    // terms: non-interacting, XC, Hartree, LPP, ions (Sigma = sum); Eq. (StressTensor)
    double S[5][9] = {};
    for (int d = 0; d < 3; ++d) {
        S[0][4 * d] = -dV * (es.PS + es.WG) / V;             // delta/V int (f_s - n v_s)
        S[1][4 * d] = -dV * es.PXC / V;                      // delta/V int n (eps_xc - v_xc)
        S[2][4 * d] = -es.EH / V;
        S[3][4 * d] = -es.Eloc / V;
        S[4][4 * d] = -o[24] / V - Ebg / V;
    }
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    for (int q = 0; q < 6; ++q) {
        const double add[5] = {-dV * o[q] / V, 0.0, o[6 + q], -2.0 * o[12 + q],
                               -0.5 / V * o[18 + q] + 2.0 / V * o[25 + q]};
        for (int t = 0; t < 5; ++t) {
            S[t][3 * ia[q] + ib[q]] += add[t];
            if (ia[q] != ib[q]) S[t][3 * ib[q] + ia[q]] += add[t];
        }
    }
    for (int k = 0; k < 9; ++k) {
        sigma[k] = S[0][k] + S[1][k] + S[2][k] + S[3][k] + S[4][k];
        if (terms)
            for (int t = 0; t < 5; ++t) terms[9 * t + k] = S[t][k];
    }
    return OFDFT_OK;
}

ofdft_status ofdft_get_density(ofdft_ctx *c, double *n)
{
    if (!c || !n) return fail(c, OFDFT_EINVAL, "NULL argument");
    NOT_BUSY(c);
    cudaSetDevice(c->dev);
    const long long N = c->g.N;
    CK(cudaMemcpyAsync(n, c->f[0].phi, N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (long long i = 0; i < N; ++i) n[i] *= n[i];
    return OFDFT_OK;
}

ofdft_status ofdft_set_masses(ofdft_ctx *c, const double *m)
{
    if (!c || !m) return fail(c, OFDFT_EINVAL, "NULL argument");
    NOT_BUSY(c);
    for (int i = 0; i < c->nat; ++i)
        if (!(m[i] > 0.0)) return fail(c, OFDFT_EINVAL, "masses must be > 0");
    c->masses.assign(m, m + c->nat);
    CK(cudaMemcpyAsync(c->Md, m, c->nat * sizeof(double), cudaMemcpyHostToDevice, c->st));
    return OFDFT_OK;
}

ofdft_status ofdft_md_step(ofdft_ctx *c, const ofdft_md_params *mp, int nsteps, double *pos, double *vel,
                           double *F, ofdft_energy *E, ofdft_stats *stats)
{
    if (!c || !mp) return fail(c, OFDFT_EINVAL, "NULL argument");
    NOT_BUSY(c);
    if (!(mp->dt_fs > 0.0) || !(mp->gtol > 0.0) || mp->maxit <= 0 || nsteps < 0)
        return fail(c, OFDFT_EINVAL, "bad MD parameters");
    cudaSetDevice(c->dev);
    const int nat = c->nat;
    FieldSet &f = c->f[0];
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
    auto add = [&](const ofdft_stats &st) {
        tot.iterations += st.iterations;
        tot.evaluations += st.evaluations;
        tot.evaluations_lo += st.evaluations_lo;
        tot.gnorm = st.gnorm;
    };
    if (!c->md_ready) {
        ofdft_stats st{};
        s = run_minimize(c, mp->gtol, mp->maxit, st, es);
        add(st);
        if (s != OFDFT_OK) {
            tot.status = s;
            if (stats) *stats = tot;
            return s;
        }
        s = forces_now(c, es);
        if (s != OFDFT_OK) return s;
        CK(cudaMemcpyAsync(c->phiprev, f.phi, c->g.N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        c->md_ready = true;
    }
    for (int step = 0; step < nsteps; ++step) {
        launch_md_a(nat, c->Md, c->Rd, c->Vd, c->Fd, c->md_dt, c->md_kT, c->md_Q, ndof, c->md_thermo, c->nh, c->st);
        c->launches++;
        s = update_ions(c);
        if (s != OFDFT_OK) return s;
        // density extrapolation phi0 = 2 phi_n - phi_{n-1} (renormalised by the minimiser)
        launch_extrap<double>(c->g.N, (const double *)f.phi, c->phiprev, (double *)f.phit, c->part, c->st);
        c->launches++;
        CK(cudaMemcpyAsync(c->phiprev, f.phi, c->g.N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(f.phi, f.phit, c->g.N * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        ofdft_stats st{};
        s = run_minimize(c, mp->gtol, mp->maxit, st, es);
        add(st);
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
    CK(cudaMemcpyAsync(c->R.data(), c->Rd, 3 * nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (E) *E = c->last;
    if (stats) *stats = tot;
    return OFDFT_OK;
}

ofdft_status ofdft_md_andersen(ofdft_ctx *c, double T_kelvin, double prob, const double *u, const double *xi,
                               int *ncoll)
{
    if (!c || !u || !xi) return fail(c, OFDFT_EINVAL, "NULL argument");
    NOT_BUSY(c);
    if (!(T_kelvin > 0.0) || !isfinite(T_kelvin) || !(prob >= 0.0 && prob <= 1.0))
        return fail(c, OFDFT_EINVAL, "Andersen collisions need T > 0 and 0 <= prob <= 1");
    const int nat = c->nat;
    int hits = 0;
    for (int i = 0; i < nat; ++i) hits += u[i] < prob;
    for (int i = 0; i < 3 * nat; ++i)
        if (!isfinite(xi[i])) return fail(c, OFDFT_EINVAL, "non-finite normal deviate");
    cudaSetDevice(c->dev);
    double *d = nullptr;
    CK(cudaMallocAsync((void **)&d, 4 * (size_t)nat * sizeof(double), c->st));
    CK(cudaMemcpyAsync(d, u, nat * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(d + nat, xi, 3 * nat * sizeof(double), cudaMemcpyHostToDevice, c->st));
    launch_andersen(nat, c->Md, c->Vd, T_kelvin * kKbHa, prob, d, d + nat, c->nh, c->st);
    c->launches++;
    CK(cudaFreeAsync(d, c->st));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaGetLastError());
    if (ncoll) *ncoll = hits;
    return OFDFT_OK;
}

ofdft_status ofdft_md_state(ofdft_ctx *c, double *pos, double *vel)
{
    if (!c) return fail(c, OFDFT_EINVAL, "NULL context");
    cudaSetDevice(c->dev);
    CK(cudaStreamSynchronize(c->st));
    if (pos) CK(cudaMemcpyAsync(pos, c->Rd, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (vel) CK(cudaMemcpyAsync(vel, c->Vd, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return OFDFT_OK;
}

ofdft_status ofdft_md_conserved(ofdft_ctx *c, double *H)
{
    if (!c || !H) return fail(c, OFDFT_EINVAL, "NULL argument");
    if (!c->last_valid) return fail(c, OFDFT_EINVAL, "no MD step has run");
    double nh[4];
    CK(cudaMemcpyAsync(nh, c->nh, sizeof(nh), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
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
    if (!c || id < 0 || id > 23 || (id & 24) == 24) return fail(c, OFDFT_EINVAL, "bad timer id");
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

ofdft_status ofdft_ffmath_eval(int op, long long count, const double *x, const double *y, double *out)
{
    if (op < 0 || op > 7 || count < 0) return OFDFT_EINVAL;
    if (count > 0 && (!x || !out || (op <= 2 && !y))) return OFDFT_EINVAL;
    for (long long i = 0; i < count; ++i) {
        const ff::f2 a = ff::from_double(x[i]);
        const ff::f2 b = op <= 2 ? ff::from_double(y[i]) : ff::f2(0.0f, 0.0f);
        ff::f2 r;
        switch (op) {
        case 0: r = ff::add(a, b); break;
        case 1: r = ff::mul(a, b); break;
        case 2: r = ff::div(a, b); break;
        case 3: r = ff::sqrt(a); break;
        case 4: r = ff::exp(a); break;
        case 5: r = ff::expm1_neg(a); break;
        case 6: r = ff::log(a); break;
        default: r = ff::rcbrt(a); break;
        }
        out[i] = ff::to_double(r);
    }
    return OFDFT_OK;
}

ofdft_status ofdft_pointwise_eval(int functional, int xc, double T_kelvin, long long count, const double *n,
                                  const double *g2, int arith, double *out, long long *n_f2)
{
    FuncParams fp = functional_params(functional);
    if (fp.kind < 0 || count < 0 || !(T_kelvin > 0.0) || (arith != OFDFT_PW_F32X2 && arith != OFDFT_PW_F64))
        return OFDFT_EINVAL;
    if (count > 0 && (!n || !g2 || !out)) return OFDFT_EINVAL;
    const std::vector<double> &tab = tfunc_table_host();
    std::vector<double> tt((size_t)kDdTabSize);
    dd_tables_fill(tab.data(), tt.data());
    const ff::f2 *tab2 = reinterpret_cast<const ff::f2 *>(tt.data() + kTfSize);
    const double temp = T_kelvin * kKbHa;
    const ff::f2 tcoef = ff::from_double(2.0 / OF_K23 * temp);
    long long used = 0;
    for (long long i = 0; i < count; ++i) {
        PwOut<double> o;
        PwF2 r;
        // the gradient as the double-float kernels see it: components; here (|grad n|, 0, 0)
        const ff::f2 gr[3] = {ff::from_double(sqrt(g2[i])), ff::f2(0.0f, 0.0f), ff::f2(0.0f, 0.0f)};
        if (arith == OFDFT_PW_F32X2 && pw_core_f2(fp, tab2, tcoef, ff::from_double(n[i]), gr, xc, r)) {
            ++used;
            o.f = ff::to_double(r.f);
            o.ts = ff::to_double(r.ts);
            o.dfdn = ff::to_double(r.dfdn);
            o.wc = g2[i] > 0.0 ? ff::to_double(r.w[0]) / sqrt(g2[i]) : 0.0;
            o.eps = ff::to_double(r.eps);
            o.vxc = ff::to_double(r.vxc);
        } else {
            o = pw_point_native<double>(fp, tt.data(), temp, n[i], g2[i], xc);
        }
        double *w = out + 6 * i;
        w[0] = o.f;
        w[1] = o.ts;
        w[2] = o.dfdn;
        w[3] = o.wc;
        w[4] = o.eps;
        w[5] = o.vxc;
    }
    if (n_f2) *n_f2 = used;
    return OFDFT_OK;
}

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
