// Allocation-free energy and potential: ofdft_energy_potential_static.
//
// Same arithmetic and kernels as ofdft_setup + ofdft_energy_potential, but all
// device scratch (half spectra, local potential, phases, reduction partials,
// twiddles, temperature table) lives in one file-scope __device__ array, so a
// call allocates nothing.  Callers that cannot allocate device memory (tight
// loops where cudaMalloc could synchronise the GPU, or programs whose device
// memory belongs to another allocator) pass their own phi and v buffers.
//
// Host code reaches the array only through the address cudaGetSymbolAddress
// returns for the current device (the symbol itself is a host-side stand-in).
// The first call on a device does that lookup and uploads the temperature
// table, under a mutex, so first calls from several host threads do not race
// on the host.  Every call reuses the same array; calls that overlap on the
// GPU race.
#include <math.h>
#include <string.h>

#include <mutex>

#include "kernels.h"
#include "pointwise.cuh"

using namespace ofdft;

namespace {

// Limits of the static path.
constexpr int kSMaxEdge = 64;
constexpr long long kSMaxN = 32768;
constexpr int kSMaxAtoms = 64;
// half spectrum: nx*ny*(nz/2+1) <= N/2 + nx*ny <= 16384 + 4096 (nz >= 8)
constexpr long long kSMaxNH = kSMaxN / 2 + kSMaxN / 8;
constexpr long long kSMaxPart = 3LL * kSMaxEdge * 5 + 15LL * (kSMaxN / 16) + 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets inside the scratch array.
constexpr size_t kOffSpec = 0;                                              // 4 spectra
constexpr size_t kSpecBytes = align256((size_t)kSMaxNH * sizeof(double2));
constexpr size_t kOffVext = kOffSpec + 4 * kSpecBytes;
constexpr size_t kOffVpart = kOffVext + kSpecBytes;
constexpr size_t kOffPhase = kOffVpart + align256((size_t)kSMaxN * sizeof(double));
constexpr size_t kPhaseBytes = align256((size_t)kSMaxAtoms * (3 * kSMaxEdge) * sizeof(double2));
constexpr size_t kOffIons = kOffPhase + kPhaseBytes;
constexpr size_t kOffZ = kOffIons + align256(3 * kSMaxAtoms * sizeof(double));
constexpr size_t kOffPart = kOffZ + align256(kSMaxAtoms * sizeof(double));
constexpr size_t kOffScal = kOffPart + align256((size_t)kSMaxPart * sizeof(double));
constexpr size_t kOffTw = kOffScal + align256(64 * sizeof(double));
constexpr size_t kOffTab = kOffTw + align256(3 * kSMaxEdge * 2 * sizeof(double2));   // + double-float copy
constexpr size_t kScratchBytes = kOffTab + align256((size_t)kDdTabSize * sizeof(double));   // + splits

static __device__ __align__(256) unsigned char g_ofdft_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DevState {
    bool ready;
    unsigned char *base;
};
DevState g_dev[kMaxDevices];
double g_tab_host[kDdTabSize];    // host temperature table + double-float tables, filled once
bool g_tab_ready = false;
std::mutex g_setup_mu;            // guards g_dev, g_tab_host and g_tab_ready (locking allocates nothing)

// Status only: the documented limits say what OFDFT_EINVAL means here.
ofdft_status serr(ofdft_status s, const char *, cudaError_t = cudaSuccess) { return s; }

#define SCK(call, what)                                            \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return serr(OFDFT_EDEVICE, what, e_); \
    } while (0)

bool edge_ok(int n)
{
    if (n < 8 || n > kSMaxEdge || (n & 1)) return false;
    for (int p : {2, 3, 5})
        while (n % p == 0) n /= p;
    return n == 1;
}


// One-time set-up on the current device: scratch address, table, smem limits.
ofdft_status device_setup(int dev, unsigned char **base)
{
    if (dev < 0 || dev >= kMaxDevices) return serr(OFDFT_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DevState &d = g_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        SCK(cudaGetSymbolAddress(&p, g_ofdft_scratch), "cudaGetSymbolAddress of the static scratch failed");
        d.base = (unsigned char *)p;
        if (!g_tab_ready) {
            static double ttab[kTfSize];
            tfunc_table_fill(ttab);
            dd_tables_fill(ttab, g_tab_host);
            g_tab_ready = true;
        }
        SCK(cudaMemcpy(d.base + kOffTab, g_tab_host, sizeof(g_tab_host), cudaMemcpyHostToDevice),
            "temperature table upload failed");
        int optin = 0;
        SCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
            "device attribute query failed");
        // leave room for the kernels' static shared memory, as ofdft_setup does
        SCK(set_field_smem_limits<double>((size_t)optin - 8192), "shared-memory limit set-up failed");
        d.ready = true;
    }
    *base = d.base;
    return OFDFT_OK;
}

// Textbook Ewald energy on the host, no heap: real-space erfc sum, reciprocal
// sum over the box of G with |G| < gcut, self and background terms.
double ewald_host(const double L[3], int nat, const double *R, const double *Z)
{
    const double pi = 3.14159265358979323846;
    double om = L[0] * L[1] * L[2];
    double a = 1.2 * sqrt(pi) * pow((double)nat / (om * om), 1.0 / 6.0);
    double rcut = 6.3 / a, gcut = 2.0 * a * 6.3;
    int ni[3], km[3];
    for (int k = 0; k < 3; ++k) {
        ni[k] = (int)ceil(rcut / L[k] + 0.5);
        km[k] = (int)ceil(gcut * L[k] / (2.0 * pi));
    }
    double E = 0.0;
    for (int I = 0; I < nat; ++I)
        for (int J = 0; J < nat; ++J) {
            double d0[3];
            for (int k = 0; k < 3; ++k) {
                d0[k] = R[3 * I + k] - R[3 * J + k];
                d0[k] -= L[k] * rint(d0[k] / L[k]);
            }
            for (int i = -ni[0]; i <= ni[0]; ++i)
                for (int j = -ni[1]; j <= ni[1]; ++j)
                    for (int k = -ni[2]; k <= ni[2]; ++k) {
                        double dx = d0[0] - i * L[0], dy = d0[1] - j * L[1], dz = d0[2] - k * L[2];
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < 1e-24 || r2 >= rcut * rcut) continue;
                        double r = sqrt(r2);
                        E += 0.5 * Z[I] * Z[J] * erfc(a * r) / r;
                    }
        }
    for (int i = -km[0]; i <= km[0]; ++i)
        for (int j = -km[1]; j <= km[1]; ++j)
            for (int k = -km[2]; k <= km[2]; ++k) {
                double gx = 2 * pi * i / L[0], gy = 2 * pi * j / L[1], gz = 2 * pi * k / L[2];
                double g2 = gx * gx + gy * gy + gz * gz;
                if (g2 == 0.0 || g2 >= gcut * gcut) continue;
                double sr = 0.0, si = 0.0;
                for (int I = 0; I < nat; ++I) {
                    double ph = gx * R[3 * I] + gy * R[3 * I + 1] + gz * R[3 * I + 2];
                    sr += Z[I] * cos(ph);
                    si += Z[I] * sin(ph);
                }
                E += 2.0 * pi / om * exp(-g2 / (4.0 * a * a)) / g2 * (sr * sr + si * si);
            }
    double z2 = 0.0, zs = 0.0;
    for (int I = 0; I < nat; ++I) {
        z2 += Z[I] * Z[I];
        zs += Z[I];
    }
    return E - a / sqrt(pi) * z2 - pi * zs * zs / (2.0 * om * a * a);
}

}  // namespace

extern "C" ofdft_status ofdft_energy_potential_static(const double cell[9], const int grid[3], int nat,
                                                      const double *ions, const double *Z, double T_kelvin,
                                                      int functional, int xc, double rc,
                                                      const double *phi_dev, double *v_dev,
                                                      ofdft_energy *E, void *stream)
{
    if (!cell || !grid || !ions || !Z || !phi_dev || !v_dev)
        return serr(OFDFT_EINVAL, "NULL argument");
    if ((((uintptr_t)phi_dev) | ((uintptr_t)v_dev)) & 15)
        return serr(OFDFT_EINVAL, "phi_dev and v_dev must be 16-byte aligned");
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (i != j && cell[3 * i + j] != 0.0) return serr(OFDFT_EINVAL, "cell is not orthorhombic");
    if (!(cell[0] > 0 && cell[4] > 0 && cell[8] > 0)) return serr(OFDFT_EINVAL, "non-positive cell edge");
    for (int a = 0; a < 3; ++a)
        if (!edge_ok(grid[a]))
            return serr(OFDFT_EINVAL, "static path: grid edges must be even, {2,3,5}-smooth, 8..64");
    long long N = (long long)grid[0] * grid[1] * grid[2];
    if (N > kSMaxN) return serr(OFDFT_EINVAL, "static path: nx*ny*nz exceeds 32768 grid points");
    if (nat <= 0 || nat > kSMaxAtoms) return serr(OFDFT_EINVAL, "static path: nat must be in 1..64");
    if (!(T_kelvin > 0.0) || !isfinite(T_kelvin) || !(rc > 0.0) || !isfinite(rc))
        return serr(OFDFT_EINVAL, "temperature and rc must be finite and > 0");
    for (int i = 0; i < nat; ++i) {   // the per-ion checks of ofdft_setup
        if (!(Z[i] > 0.0) || !isfinite(Z[i])) return serr(OFDFT_EINVAL, "ion charges must be finite and > 0");
        for (int k = 0; k < 3; ++k)
            if (!isfinite(ions[3 * i + k])) return serr(OFDFT_EINVAL, "ion positions must be finite");
    }
    FuncParams fp = functional_params(functional);
    if (fp.kind < 0) return serr(OFDFT_EINVAL, "unknown functional");
    cudaStream_t st = (cudaStream_t)stream;
    {
        // the call copies from pageable host memory and synchronises: not
        // capturable
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
            return serr(OFDFT_EINVAL, "the stream is being captured");
    }
    int dev = 0;
    SCK(cudaGetDevice(&dev), "cudaGetDevice failed");
    unsigned char *base = nullptr;
    ofdft_status s = device_setup(dev, &base);
    if (s != OFDFT_OK) return s;

    GridInfo g{};
    g.nx = grid[0];
    g.ny = grid[1];
    g.nz = grid[2];
    g.K = g.nz / 2 + 1;
    g.N = N;
    g.NH = (long long)g.nx * g.ny * g.K;
    g.Lx = cell[0];
    g.Ly = cell[4];
    g.Lz = cell[8];
    g.omega = g.Lx * g.Ly * g.Lz;
    g.dV = g.omega / (double)N;
    g.rc = rc;
    grid_reciprocal(g);
    g.dd = 1;   // double-float FFT and pointwise arithmetic, as ofdft_setup's default
    const double T = T_kelvin * 3.166811563e-6;

    // twiddles for the three axes (host stack -> scratch), binary64 then
    // double-float pairs
    double2 tw[3][kSMaxEdge];
    float twf[3][kSMaxEdge][4];
    int n3[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < n3[a]; ++m) {
            long double ang = -2.0L * 3.14159265358979323846264338327950288L * m / n3[a];
            long double cv = cosl(ang), sv = sinl(ang);
            tw[a][m] = make_double2((double)cv, (double)sv);
            twf[a][m][0] = (float)cv;
            twf[a][m][1] = (float)(cv - (long double)twf[a][m][0]);
            twf[a][m][2] = (float)sv;
            twf[a][m][3] = (float)(sv - (long double)twf[a][m][2]);
        }
    double2 *twd = (double2 *)(base + kOffTw);
    double2 *twfd = twd + 3 * kSMaxEdge;
    SCK(cudaMemcpyAsync(twd, tw, sizeof(tw), cudaMemcpyHostToDevice, st), "twiddle upload failed");
    SCK(cudaMemcpyAsync(twfd, twf, sizeof(twf), cudaMemcpyHostToDevice, st), "twiddle upload failed");
    FftAxis ax = fft_axis(g.nx, twd), ay = fft_axis(g.ny, twd + kSMaxEdge),
            az = fft_axis(g.nz, twd + 2 * kSMaxEdge, 4);   // the FP64 contexts' z schedule
    ax.twf = twfd;
    ay.twf = twfd + kSMaxEdge;
    az.twf = twfd + 2 * kSMaxEdge;
    // ions -> phases -> v_ext(G)
    double *Rd = (double *)(base + kOffIons), *Zd = (double *)(base + kOffZ);
    SCK(cudaMemcpyAsync(Rd, ions, 3 * nat * sizeof(double), cudaMemcpyHostToDevice, st), "ion upload failed");
    SCK(cudaMemcpyAsync(Zd, Z, nat * sizeof(double), cudaMemcpyHostToDevice, st), "charge upload failed");
    double2 *px = (double2 *)(base + kOffPhase);
    double2 *py = px + (size_t)nat * g.nx, *pz = py + (size_t)nat * g.ny;
    double2 *vext = (double2 *)(base + kOffVext);
    launch_phases(g, nat, Rd, px, py, pz, nullptr, st);
    launch_vext(g, nat, Zd, px, py, pz, nullptr, vext, st);

    // evaluation (same kernel sequence as the context path)
    const size_t specN = kSpecBytes / sizeof(double2);
    double2 *s0 = (double2 *)(base + kOffSpec), *s1 = s0 + specN, *s2 = s1 + specN, *s3 = s2 + specN;
    const double *tab = (const double *)(base + kOffTab);
    double *vpart = (double *)(base + kOffVpart);
    double *part = (double *)(base + kOffPart), *scal = (double *)(base + kOffScal);
    SCK(cudaMemsetAsync(scal, 0, 64 * sizeof(double), st), "scalar clear failed");
    const int nbx = xpass_blocks(g);
    const long long npairs = (long long)g.nx * g.ny / 2;
    double *pA = part, *pB = pA + 3 * nbx, *pC = pB + 6 * npairs;
    double *ph = const_cast<double *>(phi_dev);
    const bool fttf = fp.kind == 0;
    // the second to fourth spectra double as real fields (2 NH >= N values):
    // derivatives of n, then the fields whose derivatives make up div W;
    // v_dev holds d_x U_x + d_y U_y until the final pass overwrites it with v
    double *d0 = (double *)s1, *d1 = (double *)s2, *d2 = (double *)s3;
    launch_zfwd<double>(g, az, 1, nullptr, ph, nullptr, 0.0, 0.0, nullptr, nullptr, s0, st, fttf ? nullptr : d2);
    launch_ypass<double>(g, ay, false, s0, 1, specN, st);
    launch_xhl<double>(g, ax, s0, vext, nullptr, 1, pA, st);
    launch_ypass<double>(g, ay, true, s0, 1, specN, st);
    int nbz, nbg = 0;   // blocks of the final z pass and of the pointwise stage: their partial sums
    if (fttf) {
        nbz = launch_zfinal<double>(g, az, true, s0, nullptr, ph, nullptr, nullptr, 1.0, 0.0, nullptr, T, fp,
                                    tab, xc, v_dev, pC, st);
    } else {
        launch_dline<double>(g, ax, 0, 0, 0, ph, d0, st);
        launch_dline<double>(g, ay, 1, 0, 0, ph, d1, st);
        nbg = launch_pw<double>(g, d0, d1, d2, ph, T, fp, tab, xc, vpart, pB, false, st);
        launch_dline<double>(g, ax, 0, 1, 0, d0, v_dev, st);
        launch_dline<double>(g, ay, 1, 1, 1, d1, v_dev, st);
        nbz = launch_zfinal_gga<double>(g, az, s0, d2, vpart, v_dev, nullptr, ph, nullptr, nullptr, 1.0, 0.0,
                                        nullptr, v_dev, pC, st);
    }
    launch_reduce_eval(pA, nbx, pB, nbg, pC, nbz, !fttf, scal, st);
    double h[18];
    SCK(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, st), "scalar read-back failed");
    SCK(cudaStreamSynchronize(st), "stream synchronisation failed");
    SCK(cudaGetLastError(), "kernel launch failed");

    const double *f = fttf ? h + 9 : h + 3;
    const double dV = g.dV, om = g.omega;
    double L[3] = {g.Lx, g.Ly, g.Lz};
    double Ne = 0.0, zs = 0.0;
    for (int i = 0; i < nat; ++i) {
        Ne += Z[i];
        zs += 3.14159265358979323846 * Z[i] * rc * rc;
    }
    double E_ion = ewald_host(L, nat, ions, Z);
    ofdft_energy e;
    memset(&e, 0, sizeof(e));
    e.F_s = dV * f[0];
    e.minus_TS = -dV * f[1];
    e.E_H = h[0];
    e.E_loc = h[1];
    e.F_xc = dV * f[2];
    e.E_ion = E_ion;
    e.F_tot = e.F_s + e.E_H + e.E_loc + e.F_xc + e.E_ion;
    e.E_int = e.F_tot + dV * f[1];
    e.mu = h[15] / h[16];
    e.E_alphaZ = Ne * zs / om;
    e.P_s = (dV * f[3] + (4.0 / 3.0) * dV * (fttf ? 0.0 : f[4])) / om;
    e.P_xc = dV * f[5] / om;
    e.P_H = h[0] / (3.0 * om);
    e.P_loc = h[2];
    e.P_ion = E_ion / (3.0 * om);
    e.P = e.P_s + e.P_xc + e.P_H + e.P_loc + e.P_ion;
    if (!isfinite(e.F_tot + e.mu)) return serr(OFDFT_ENUMERIC, "non-finite energy or potential");
    if (E) *E = e;
    return OFDFT_OK;
}
