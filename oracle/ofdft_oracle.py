"""Oracle (TEST INFRASTRUCTURE ONLY): finite-T orbital-free DFT in plain FP64.

Written from arXiv:1406.0835 (Karasiev, Sjostrom, Trickey), section by
section; each function names the equation it follows.  Only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU-baseline legs may use it.
It shares no code with the CUDA library and imports nothing from it.

Discretisation (a reading; the paper works in the continuum): integrals are
dV * sum over a periodic grid (orthorhombic, or a general cell through
CellGrid); n(G) = fftn(n)/N over the full FFT box with integer wave numbers
k in {-n/2+1, ..., n/2}.  Even-order operators
(G^2, Hartree, local pseudopotential) use k = +n/2 on a Nyquist plane and the
real part of the inverse transform; first derivatives i G_a are zeroed on the
a-Nyquist plane, so gradient and divergence are exact adjoints and the
potential is the exact derivative of the discrete free energy.

Units: Hartree atomic units; temperatures at the interface in kelvin.
"""
import ctypes
import math

import numpy as np

from . import build as _build

# ---------------------------------------------------------------- constants
KB_HA_PER_K = 3.166811563e-6          # Boltzmann constant, hartree / kelvin
C_TF = 0.3 * (3.0 * math.pi ** 2) ** (2.0 / 3.0)   # Eq. (tauTFdefn)
AMU_ME = 1822.888486209               # atomic mass unit / electron mass
FS_AU = 41.341373335                  # femtosecond in atomic time units

# ------------------------------------------------------- Fermi-Dirac (C part)
_lib = None
_P = ctypes.POINTER(ctypes.c_double)


def _c():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        for name in ("oracle_fd_moments", "oracle_eta_of_t", "oracle_kappa_h"):
            getattr(_lib, name).argtypes = [ctypes.c_long, _P, _P]
            getattr(_lib, name).restype = ctypes.c_int
    return _lib


def fd_moments(eta):
    """I_{-1/2}, I_{1/2}, I_{3/2}, I'_{-1/2}, I''_{-1/2}, I'''_{-1/2} at eta."""
    eta = np.ascontiguousarray(eta, dtype=np.float64)
    out = np.empty(eta.shape + (6,))
    _c().oracle_fd_moments(eta.size, eta.ctypes.data_as(_P), out.ctypes.data_as(_P))
    return out


def eta_of_t(t):
    """eta solving I_{1/2}(eta) = (2/3) t^{-3/2} (Eq. (tred) with n of the ideal gas)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.empty(t.shape)
    _c().oracle_eta_of_t(t.size, t.ctypes.data_as(_P), out.ctypes.data_as(_P))
    return out


def kappa_h(t):
    """Per t: eta, kappa, kappa', kappa'', h~, h~', h~'' (footnote a of Table I).

    Returned as a tuple of arrays shaped like t.
    """
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.empty(t.shape + (7,))
    _c().oracle_kappa_h(t.size, t.ctypes.data_as(_P), out.ctypes.data_as(_P))
    return tuple(out[..., k] for k in range(7))


def xi_zeta(t):
    """xi = kappa - t kappa', zeta = -t kappa' (Eq. (xizeta)) and t-derivatives."""
    _, kap, dk, d2k, h, dh, d2h = kappa_h(t)
    xi = kap - t * dk
    zeta = -t * dk
    dxi = -t * d2k
    dzeta = -dk - t * d2k
    return dict(kappa=kap, dkappa=dk, xi=xi, zeta=zeta, dxi=dxi, dzeta=dzeta,
                h=h, dh=dh, d2h=d2h)


# ------------------------------------------------------------- grid & cell
class Grid:
    """Periodic orthorhombic grid, C order [ix][iy][iz] with iz fastest."""

    def __init__(self, L, shape):
        self.L = np.asarray(L, dtype=np.float64).reshape(3)
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.omega = float(np.prod(self.L))
        self.dV = self.omega / self.N
        kint = []
        for n in self.shape:
            k = np.fft.fftfreq(n, 1.0 / n)
            if n % 2 == 0:
                k[n // 2] = n // 2          # Nyquist taken as +n/2
            kint.append(k)
        self.kint = kint
        g1 = [2.0 * math.pi * kint[a] / self.L[a] for a in range(3)]
        self.Gx = g1[0][:, None, None]
        self.Gy = g1[1][None, :, None]
        self.Gz = g1[2][None, None, :]
        self.G2 = self.Gx ** 2 + self.Gy ** 2 + self.Gz ** 2
        # first-derivative multipliers with the a-Nyquist plane zeroed
        gd = []
        for a in range(3):
            g = g1[a].copy()
            n = self.shape[a]
            if n % 2 == 0:
                g[n // 2] = 0.0
            gd.append(g)
        self.Dx = gd[0][:, None, None]
        self.Dy = gd[1][None, :, None]
        self.Dz = gd[2][None, None, :]

    def to_G(self, f):
        """n(G) = (1/N) sum_j f_j exp(-i G.r_j)."""
        return np.fft.fftn(f) / self.N

    def to_r(self, fG):
        """Real part of sum_G f(G) exp(i G.r_j)."""
        return np.real(np.fft.ifftn(fG)) * self.N

    def grad(self, f):
        fG = self.to_G(f)
        return np.stack([self.to_r(1j * D * fG) for D in (self.Dx, self.Dy, self.Dz)])

    def div(self, W):
        acc = 1j * self.Dx * self.to_G(W[0])
        acc = acc + 1j * self.Dy * self.to_G(W[1])
        acc = acc + 1j * self.Dz * self.to_G(W[2])
        return self.to_r(acc)

    def integrate(self, f):
        return self.dV * float(np.sum(f))


class CellGrid(Grid):
    """Periodic grid of a general (triclinic) cell: rows of `cell` are the
    lattice vectors a_1..a_3 (bohr), grid point (i, j, k) sits at
    (i/n1) a_1 + (j/n2) a_2 + (k/n3) a_3.  G = k_1 b_1 + k_2 b_2 + k_3 b_3
    with a_i . b_j = 2 pi delta_ij and the same integer wave numbers and
    Nyquist conventions as the orthorhombic grid (a first derivative is
    zeroed where its own integer k_a sits on the a-Nyquist plane)."""

    def __init__(self, cell, shape):
        self.cell = np.asarray(cell, dtype=np.float64).reshape(3, 3)
        self.L = None
        self.shape = tuple(int(n) for n in shape)
        self.N = int(np.prod(self.shape))
        self.omega = abs(float(np.linalg.det(self.cell)))
        self.dV = self.omega / self.N
        self.B = 2.0 * math.pi * np.linalg.inv(self.cell).T     # rows b_j
        kint, kd = [], []
        for n in self.shape:
            k = np.fft.fftfreq(n, 1.0 / n)
            if n % 2 == 0:
                k[n // 2] = n // 2
            d = k.copy()
            if n % 2 == 0:
                d[n // 2] = 0.0
            kint.append(k)
            kd.append(d)
        self.kint = kint
        sh = [(-1, 1, 1), (1, -1, 1), (1, 1, -1)]

        def cart(ks):
            return [sum(ks[j].reshape(sh[j]) * self.B[j, a] for j in range(3)) for a in range(3)]
        self.Gx, self.Gy, self.Gz = cart(kint)
        self.G2 = self.Gx ** 2 + self.Gy ** 2 + self.Gz ** 2
        self.Dx, self.Dy, self.Dz = cart(kd)


# --------------------------------------------- enhancement factors (Sec. III B)
def F_sga(mu):
    """Eq. (SGA-F): F_tau = 1 + mu x with x = s_tau^2 (mu = 5/27 SGA, 5/3 VWTF)."""
    def F(x):
        return 1.0 + mu * x, np.full_like(x, mu)
    return F


def F_kst2(C1, a1):
    """Eq. (KST2F): F_tau = 1 + C1 x / (1 + a1 x)."""
    def F(x):
        den = 1.0 + a1 * x
        return 1.0 + C1 * x / den, C1 / den ** 2
    return F


def F_vt84f(x, mu=2.778, alpha=1.2965):
    """Eq. (VT84F) with m = 8, n = 4 written in x = s^2 (s^{m/2} = x^2, s^{-n/2} = 1/x).

    F = 1 - mu x e^{-alpha x}/(1 + mu x) + (1 - e^{-alpha x^2})(1/x - 1) + (5/3) x.
    Reading: the removable 0/0 at x = 0 takes its limit F = 1,
    dF/dx = -mu + alpha + 5/3.
    """
    x = np.asarray(x, dtype=np.float64)
    xs = np.where(x > 0.0, x, 1.0)
    e1 = np.exp(-alpha * xs)
    em = -np.expm1(-alpha * xs * xs)                 # 1 - exp(-alpha x^2)
    den = 1.0 + mu * xs
    F = 1.0 - mu * xs * e1 / den + em * (1.0 / xs - 1.0) + (5.0 / 3.0) * xs
    dF = (-mu * e1 * (1.0 - alpha * xs - alpha * mu * xs * xs) / den ** 2
          + 2.0 * alpha * (1.0 - em) * (1.0 - xs) - em / (xs * xs) + 5.0 / 3.0)
    F = np.where(x > 0.0, F, 1.0)
    dF = np.where(x > 0.0, dF, -mu + alpha + 5.0 / 3.0)
    return F, dF


FUNCTIONALS = {
    "fttf": None,
    "sga": F_sga(5.0 / 27.0),
    "vwtf": F_sga(5.0 / 3.0),
    "vt84f": F_vt84f,
    "kst2": F_kst2(2.03087, 0.29424),
    "tw": F_kst2(0.2319, 0.2748),
    "apbef": F_kst2(0.23889, 0.23889 / 0.804),
}


# ------------------------------------------- non-interacting free energy
def reduced_t(n, T):
    """Eq. (tred): t = 2 T / (3 pi^2 n)^{2/3}."""
    return 2.0 * T / (3.0 * math.pi ** 2 * n) ** (2.0 / 3.0)


def fs_fttf(n, T):
    """Finite-T Thomas-Fermi: f = tau0 kappa (Eq. (fTF)), v by Eq. (vTF).

    Returns dict with f, dfdn, f_kin = tau0 xi (internal), f_ent = tau0 zeta (T s).
    """
    tau0 = C_TF * n ** (5.0 / 3.0)
    dtau0 = (5.0 / 3.0) * C_TF * n ** (2.0 / 3.0)
    t = reduced_t(n, T)
    dtdn = -2.0 * t / (3.0 * n)
    z = xi_zeta(t)
    f = tau0 * z["kappa"]
    v = dtau0 * z["kappa"] + tau0 * z["dkappa"] * dtdn
    return dict(f=f, dfdn=v, f_kin=tau0 * z["xi"], f_ent=tau0 * z["zeta"],
                W=None)


def fs_gga(n, gradn, T, Fenh):
    """Generic finite-T GGA, Eqs. (FGGA), (xizeta), (s_s), (s_0defn), (vftGGA).

    f = tau0 xi F_tau(s_tau^2) - tau0 zeta F_sigma(s_sigma^2), F_sigma = 2 - F_tau.
    The sigma terms of Eq. (vftGGA) are all taken with a minus sign (the exact
    derivative of Eq. (FGGA)); W = df/d(grad n) is the argument of the
    divergence in its last line.
    """
    tau0 = C_TF * n ** (5.0 / 3.0)
    dtau0 = (5.0 / 3.0) * C_TF * n ** (2.0 / 3.0)
    t = reduced_t(n, T)
    dtdn = -2.0 * t / (3.0 * n)
    z = xi_zeta(t)
    xi, zeta, dxi, dzeta = z["xi"], z["zeta"], z["dxi"], z["dzeta"]
    h, dh, d2h = z["h"], z["dh"], z["d2h"]
    g2 = np.sum(gradn * gradn, axis=0)
    cs = 1.0 / (4.0 * (3.0 * math.pi ** 2) ** (2.0 / 3.0) * n ** (8.0 / 3.0))
    s2 = g2 * cs                                   # Eq. (s_0defn) squared
    A = (h - t * dh) / xi                          # s_tau^2 = s^2 A (Eq. (s_s))
    B = t * dh / zeta                              # s_sigma^2 = s^2 B
    dA = -t * d2h / xi - (h - t * dh) * dxi / xi ** 2
    dB = (dh + t * d2h) / zeta - t * dh * dzeta / zeta ** 2
    x_t = s2 * A
    x_s = s2 * B
    Ft, dFt = Fenh(x_t)
    Fs_tau, dFs_tau = Fenh(x_s)
    Fs, dFs = 2.0 - Fs_tau, -dFs_tau               # F_sigma = 2 - F_tau(s_sigma)
    f_kin = tau0 * xi * Ft
    f_ent = tau0 * zeta * Fs
    f = f_kin - f_ent
    dxt_dn = -(8.0 / 3.0) * x_t / n
    dxs_dn = -(8.0 / 3.0) * x_s / n
    dxt_dt = s2 * dA
    dxs_dt = s2 * dB
    dfdn = (dtau0 * xi * Ft + tau0 * dxi * dtdn * Ft
            + tau0 * xi * dFt * (dxt_dn + dxt_dt * dtdn)
            - dtau0 * zeta * Fs - tau0 * dzeta * dtdn * Fs
            - tau0 * zeta * dFs * (dxs_dn + dxs_dt * dtdn))
    coef = (tau0 * xi * dFt * A - tau0 * zeta * dFs * B) * 2.0 * cs
    W = coef[None] * gradn
    return dict(f=f, dfdn=dfdn, f_kin=f_kin, f_ent=f_ent, W=W)


# ------------------------------------------------------------- XC (Sec. IV)
def _pz81_constants():
    """PZ81 correlation constants.  gamma, beta1, beta2, A, B as published;
    C and D from the two conditions the parametrisation was built on: eps_c
    and d eps_c/d r_s continuous at r_s = 1 (the published C = 0.0020,
    D = -0.0116 are these values rounded, and the rounding leaves a 3e-5 Ha
    jump in eps_c at r_s = 1 that stalls the minimiser near that density)."""
    g, b1, b2, A, B = -0.1423, 1.0529, 0.3334, 0.0311, -0.048
    den = 1.0 + b1 + b2
    e1 = g / den                                   # Pade branch at r_s = 1
    de1 = -g * (0.5 * b1 + b2) / den ** 2          # its r_s derivative
    D = e1 - B                                     # A ln 1 + B + C 0 + D = e1
    C = de1 - A - D                                # A + C (ln 1 + 1) + D = de1
    return dict(gamma=g, beta1=b1, beta2=b2, A=A, B=B, C=C, D=D)


PZ = _pz81_constants()
EX_COEF = 0.75 * (3.0 / math.pi) ** (1.0 / 3.0)   # eps_x = -EX_COEF n^{1/3}


def pz81(n):
    """Perdew-Zunger 1981 unpolarised LDA (cited in Sec. IV, used for all timings).

    eps_xc = eps_x + eps_c(r_s); v_xc = eps_xc + n d eps_xc/dn with
    dr_s/dn = -r_s/(3n) (Eq. (vxc1) at T = 0).  Reading: r_s >= 1 takes the
    Pade branch; C and D make both branches meet with equal value and slope
    (see _pz81_constants).  Returns eps_xc, v_xc.
    """
    rs = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    ex = -EX_COEF * n ** (1.0 / 3.0)
    dex = -ex / rs                                  # d eps_x / d r_s (eps_x ~ 1/r_s)
    hi = rs >= 1.0
    r = np.where(hi, rs, 1.0)
    sq = np.sqrt(r)
    den = 1.0 + PZ["beta1"] * sq + PZ["beta2"] * r
    ec_hi = PZ["gamma"] / den
    dec_hi = -PZ["gamma"] * (PZ["beta1"] / (2.0 * sq) + PZ["beta2"]) / den ** 2
    rl = np.where(hi, 0.5, rs)
    lr = np.log(rl)
    ec_lo = PZ["A"] * lr + PZ["B"] + PZ["C"] * rl * lr + PZ["D"] * rl
    dec_lo = PZ["A"] / rl + PZ["C"] * (lr + 1.0) + PZ["D"]
    ec = np.where(hi, ec_hi, ec_lo)
    dec = np.where(hi, dec_hi, dec_lo)
    eps = ex + ec
    v = eps - rs / 3.0 * (dex + dec)
    return eps, v


# -------------------------------------------- local pseudopotential (Sec. V A)
def lpp_form(G2, omega, rc):
    """Gaussian-ion local pseudopotential per unit charge:
    w(G) = -4 pi exp(-G^2 rc^2 / 4) / (Omega G^2), G = 0 dropped
    (the Fourier transform of -erf(r/rc)/r)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        w = -4.0 * math.pi * np.exp(-G2 * rc * rc / 4.0) / (omega * G2)
    w[G2 == 0.0] = 0.0
    return w


# Heine-Abarenkov hydrogen LPP, Eq. (E4A): parameters printed for H.
HA_H = dict(rc=0.25, A=6.18, qc=29.97)


def lpp_form_ha(G2, omega, Z, rc, A, qc):
    """Heine-Abarenkov local pseudopotential of one ion, Eq. (E4A):
    w(q) = -4 pi/(Omega q^2) [(Z - A rc) cos(q rc) + (A/q) sin(q rc)] f(q),
    f(q) = exp(-(q/qc)^6), q = |G|, G = 0 dropped.  Not proportional to Z."""
    q = np.sqrt(G2)
    with np.errstate(divide="ignore", invalid="ignore"):
        B = (Z - A * rc) * np.cos(q * rc) + (A / q) * np.sin(q * rc)
        w = -4.0 * math.pi * B * np.exp(-(q / qc) ** 6) / (omega * G2)
    w[G2 == 0.0] = 0.0
    return w


def lpp_pform_ha(G2, omega, Z, rc, A, qc):
    """Volume-derivative weight of Eq. (E4A) for the pressure: the LPP term is
    sum_G Re[n*(G) sum_I wp_I(G) e^{-iG.R_I}] with wp = w + (q/3) dw/dq
    (Omega w(q) depends on the cell only through q; Omega n(G) and the
    fractional coordinates are fixed under a uniform dilation)."""
    q = np.sqrt(G2)
    with np.errstate(divide="ignore", invalid="ignore"):
        s, c = np.sin(q * rc), np.cos(q * rc)
        B = (Z - A * rc) * c + (A / q) * s
        dB = -(Z - A * rc) * rc * s + A * (rc * c / q - s / (q * q))   # dB/dq
        f = np.exp(-(q / qc) ** 6)
        df = -6.0 * q ** 5 / qc ** 6 * f                              # df/dq
        w = -4.0 * math.pi * B * f / (omega * G2)
        dw = -4.0 * math.pi / omega * ((dB * f + B * df) / G2 - 2.0 * B * f / (G2 * q))
        wp = w + q * dw / 3.0
    wp[G2 == 0.0] = 0.0
    return wp


def alpha_z_ha(Z, rc, A):
    """G -> 0 limit of Omega w(q) + 4 pi Z/q^2 for Eq. (E4A): the integral of
    v(r) + Z/r over the core of the model (v = -A inside rc, -Z/r outside)."""
    return 2.0 * math.pi * Z * rc * rc - 4.0 * math.pi / 3.0 * A * rc ** 3


def structure_phase(grid, R):
    """exp(-i G.R) on the full box (separable in x, y, z), + Nyquist convention."""
    return (np.exp(-1j * grid.Gx * R[0]) * np.exp(-1j * grid.Gy * R[1])
            * np.exp(-1j * grid.Gz * R[2]))


def lpp_vG(grid, R, Z, rc):
    """v_ext(G) = sum_I Z_I w(G) exp(-i G.R_I) on the full box."""
    w = lpp_form(grid.G2, grid.omega, rc)
    vG = np.zeros(grid.shape, dtype=np.complex128)
    for I in range(len(Z)):
        vG += Z[I] * w * structure_phase(grid, R[I])
    return vG


def lpp_vG_ha(grid, R, Z, rc, A, qc, form=lpp_form_ha):
    """v_ext(G) = sum_I w_I(G) exp(-i G.R_I) with the Eq. (E4A) form of each
    ion (form=lpp_pform_ha gives the pressure weights instead)."""
    vG = np.zeros(grid.shape, dtype=np.complex128)
    for I in range(len(Z)):
        vG += form(grid.G2, grid.omega, Z[I], rc, A, qc) * structure_phase(grid, R[I])
    return vG


# ------------------------------------------------------------------ Ewald
def ewald(L, R, Z, alpha=None):
    """Ion-ion energy E_ion of Eq. (E1) by the textbook Ewald sum.

    E = 1/2 sum'_{I,J,L} Z_I Z_J erfc(a r)/r + (2 pi/Omega) sum_{G!=0}
        exp(-G^2/4a^2)/G^2 |S(G)|^2 - a/sqrt(pi) sum Z^2 - pi (sum Z)^2/(2 Omega a^2).
    Returns (E, forces [nat,3]).  Pressure is E/(3 Omega) (Coulomb scaling).
    """
    from scipy.special import erfc
    L = np.asarray(L, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    Z = np.asarray(Z, dtype=np.float64)
    nat = len(Z)
    omega = float(np.prod(L))
    if alpha is None:
        alpha = math.sqrt(math.pi) * (nat / omega ** 2) ** (1.0 / 6.0)
    rcut = 6.5 / alpha
    gcut = 2.0 * alpha * 6.5
    # real space
    E = 0.0
    F = np.zeros((nat, 3))
    nimg = [int(math.ceil(rcut / L[a])) + 1 for a in range(3)]
    shifts = np.array([(i, j, k) for i in range(-nimg[0], nimg[0] + 1)
                       for j in range(-nimg[1], nimg[1] + 1)
                       for k in range(-nimg[2], nimg[2] + 1)], dtype=np.float64) * L
    for I in range(nat):
        d = R[I][None, None, :] - R[None, :, :] - shifts[:, None, :]   # [img, J, 3]
        r = np.sqrt(np.sum(d * d, axis=2))
        mask = (r > 1e-12) & (r < rcut)
        rr = np.where(mask, r, 1.0)
        zz = Z[I] * Z[None, :]
        e = np.where(mask, zz * erfc(alpha * rr) / rr, 0.0)
        E += 0.5 * float(np.sum(e))
        fmag = np.where(mask, zz * (erfc(alpha * rr) / rr ** 2
                                    + 2.0 * alpha / math.sqrt(math.pi)
                                    * np.exp(-(alpha * rr) ** 2) / rr), 0.0)
        F[I] += np.sum(fmag[:, :, None] * d / rr[:, :, None], axis=(0, 1))
    # reciprocal space
    km = [int(math.ceil(gcut * L[a] / (2.0 * math.pi))) for a in range(3)]
    kx = np.arange(-km[0], km[0] + 1)
    ky = np.arange(-km[1], km[1] + 1)
    kz = np.arange(-km[2], km[2] + 1)
    K = np.array(np.meshgrid(kx, ky, kz, indexing="ij")).reshape(3, -1).T
    G = 2.0 * math.pi * K / L
    G2 = np.sum(G * G, axis=1)
    sel = (G2 > 0) & (G2 < gcut * gcut)
    G = G[sel]
    G2 = G2[sel]
    wG = np.exp(-G2 / (4.0 * alpha * alpha)) / G2
    ph = np.exp(1j * (G @ R.T))                    # [nG, nat] = exp(i G.R_I)
    S = ph @ Z
    E += (2.0 * math.pi / omega) * float(np.sum(wG * np.abs(S) ** 2))
    F += (4.0 * math.pi / omega) * Z[:, None] * (
        (wG[:, None] * np.imag(np.conj(S)[:, None] * ph)).T @ G)
    E -= alpha / math.sqrt(math.pi) * float(np.sum(Z * Z))
    E -= math.pi * float(np.sum(Z)) ** 2 / (2.0 * omega * alpha * alpha)
    return E, F


def ewald_cell(cell, R, Z, alpha=None):
    """Ewald sum of Eq. (E1)'s E_ion for a general cell (rows = lattice
    vectors), with forces and the stress tensor
    Sigma_ab = (1/Omega) dE/d eps_ab at fixed fractional coordinates:
      real space   -(1/2 Omega) sum' Z_I Z_J [erfc(a r)/r + (2a/sqrt pi) e^{-a^2 r^2}] r_a r_b / r^2,
      reciprocal   -delta_ab E_G/Omega + (4 pi/Omega^2) sum_{G!=0} |S|^2 e^{-G^2/4a^2}/G^2
                   (1/(4a^2) + 1/G^2) G_a G_b,
      background   -delta_ab E_bg/Omega  (E_bg = -pi (sum Z)^2/(2 Omega a^2));
    the self term does not depend on the cell.  Returns (E, F [nat,3], Sigma [3,3])."""
    from scipy.special import erfc
    A = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    Z = np.asarray(Z, dtype=np.float64)
    nat = len(Z)
    omega = abs(float(np.linalg.det(A)))
    B = 2.0 * math.pi * np.linalg.inv(A).T
    if alpha is None:
        alpha = math.sqrt(math.pi) * (nat / omega ** 2) ** (1.0 / 6.0)
    rcut = 6.5 / alpha
    gcut = 2.0 * alpha * 6.5
    E = 0.0
    F = np.zeros((nat, 3))
    S = np.zeros((3, 3))
    # real space: lattice planes a_i are 2 pi/|b_i| apart
    nimg = [int(math.ceil(rcut * np.linalg.norm(B[i]) / (2.0 * math.pi))) + 1 for i in range(3)]
    n = np.array([(i, j, k) for i in range(-nimg[0], nimg[0] + 1)
                  for j in range(-nimg[1], nimg[1] + 1)
                  for k in range(-nimg[2], nimg[2] + 1)], dtype=np.float64)
    shifts = n @ A
    for I in range(nat):
        d = R[I][None, None, :] - R[None, :, :] - shifts[:, None, :]
        r = np.sqrt(np.sum(d * d, axis=2))
        mask = (r > 1e-12) & (r < rcut)
        rr = np.where(mask, r, 1.0)
        zz = Z[I] * Z[None, :]
        e = np.where(mask, zz * erfc(alpha * rr) / rr, 0.0)
        E += 0.5 * float(np.sum(e))
        g = np.where(mask, zz * (erfc(alpha * rr) / rr
                                 + 2.0 * alpha / math.sqrt(math.pi) * np.exp(-(alpha * rr) ** 2)), 0.0)
        F[I] += np.sum((g / rr ** 2)[:, :, None] * d, axis=(0, 1))
        S -= 0.5 / omega * np.einsum("ij,ija,ijb->ab", g / rr ** 2, d, d)
    # reciprocal space
    km = [int(math.ceil(gcut * np.linalg.norm(A[i]) / (2.0 * math.pi))) for i in range(3)]
    K = np.array(np.meshgrid(*[np.arange(-m, m + 1) for m in km], indexing="ij")).reshape(3, -1).T
    G = K @ B
    G2 = np.sum(G * G, axis=1)
    sel = (G2 > 0) & (G2 < gcut * gcut)
    G, G2 = G[sel], G2[sel]
    wG = np.exp(-G2 / (4.0 * alpha * alpha)) / G2
    ph = np.exp(1j * (G @ R.T))
    SG = ph @ Z
    S2 = np.abs(SG) ** 2
    EG = (2.0 * math.pi / omega) * float(np.sum(wG * S2))
    E += EG
    F += (4.0 * math.pi / omega) * Z[:, None] * ((wG[:, None] * np.imag(np.conj(SG)[:, None] * ph)).T @ G)
    c = S2 * wG * (1.0 / (4.0 * alpha * alpha) + 1.0 / G2)
    S += -EG / omega * np.eye(3) + (4.0 * math.pi / omega ** 2) * np.einsum("g,ga,gb->ab", c, G, G)
    E -= alpha / math.sqrt(math.pi) * float(np.sum(Z * Z))
    Ebg = -math.pi * float(np.sum(Z)) ** 2 / (2.0 * omega * alpha * alpha)
    E += Ebg
    S += -Ebg / omega * np.eye(3)
    return E, F, S


# -------------------------------------------------------------- the system
class System:
    """Cell, ions, grid, temperature and functional choice (Sec. II, V C).

    ions: Cartesian bohr [nat,3]; Z: valence charges; T_kelvin (keyword TEMP).
    """

    def __init__(self, L, shape, ions, Z, T_kelvin, functional="fttf",
                 rc=0.25, xc=True, lpp="gauss", ha_A=HA_H["A"], ha_qc=HA_H["qc"], cell=None):
        if lpp not in ("gauss", "ha"):
            raise ValueError("lpp must be 'gauss' or 'ha'")
        self.lpp = lpp
        self.ha_A = float(ha_A)
        self.ha_qc = float(ha_qc)
        # cell: lattice vectors as rows for a general cell (L is then unused)
        self.cell = None if cell is None else np.asarray(cell, dtype=np.float64).reshape(3, 3)
        self.grid = Grid(L, shape) if cell is None else CellGrid(cell, shape)
        self.R = np.array(ions, dtype=np.float64).reshape(-1, 3)
        self.Z = np.array(Z, dtype=np.float64).reshape(-1)
        self.T = float(T_kelvin) * KB_HA_PER_K
        self.functional = functional
        self.rc = float(rc)
        self.xc = xc
        self.Ne = float(np.sum(self.Z))
        self.set_positions(self.R)

    def set_positions(self, R):
        self.R = np.array(R, dtype=np.float64).reshape(-1, 3)
        if self.lpp == "ha":
            args = (self.grid, self.R, self.Z, self.rc, self.ha_A, self.ha_qc)
            self.vG = lpp_vG_ha(*args)
            self.vpG = lpp_vG_ha(*args, form=lpp_pform_ha)
        else:
            self.vG = lpp_vG(self.grid, self.R, self.Z, self.rc)
        self.v_ext = self.grid.to_r(self.vG)
        if self.cell is None:
            self.E_ion, self.F_ion = ewald(self.grid.L, self.R, self.Z)
        else:
            self.E_ion, self.F_ion, _ = ewald_cell(self.cell, self.R, self.Z)

    def uniform_phi(self):
        return np.full(self.grid.shape, math.sqrt(self.Ne / self.grid.omega))


def evaluate(sys, phi):
    """Free energy F_tot[n] (Eq. (E1) with the constraint term left out) and
    its functional derivative v = dF/dn at n = phi^2, plus the pressure terms.

    F_tot = F_s + F_H + F_xc + int n v_ext + E_ion  (Eqs. (E1)-(E4), (E2)).
    """
    g = sys.grid
    n = phi * phi
    nG = g.to_G(n)
    with np.errstate(divide="ignore", invalid="ignore"):
        kH = 4.0 * math.pi / g.G2
    kH[g.G2 == 0.0] = 0.0
    vHG = kH * nG
    vH = g.to_r(vHG)
    E_H = 0.5 * g.integrate(n * vH)                                  # Eq. (E2)
    E_loc = g.integrate(n * sys.v_ext)
    fun = FUNCTIONALS[sys.functional]
    if fun is None:
        fs = fs_fttf(n, sys.T)
        gradn = None
        W = None
        v_s = fs["dfdn"]
        WdotG = 0.0
    else:
        gradn = g.grad(n)
        fs = fs_gga(n, gradn, sys.T, fun)
        W = fs["W"]
        v_s = fs["dfdn"] - g.div(fs["W"])                            # Eq. (vftGGA)
        WdotG = g.integrate(np.sum(fs["W"] * gradn, axis=0))
    F_s = g.integrate(fs["f"])
    TS = g.integrate(fs["f_ent"])
    if sys.xc:
        eps, vxc = pz81(n)
        F_xc = g.integrate(n * eps)
        P_xc = g.integrate(n * (vxc - eps)) / g.omega               # Eq. (stressLSDAxc)
    else:
        eps = vxc = np.zeros_like(n)
        F_xc = 0.0
        P_xc = 0.0
    v = v_s + vH + sys.v_ext + vxc
    F_el = F_s + E_H + E_loc + F_xc
    F_tot = F_el + sys.E_ion
    # pressure: P = -(1/3) Tr Sigma (Eq. (pressure)), term by term
    P_s = (g.integrate(n * v_s - fs["f"]) + WdotG / 3.0) / g.omega  # Eqs. (stressTF_a,b)
    P_H = E_H / (3.0 * g.omega)
    if sys.lpp == "ha":
        P_loc = float(np.real(np.sum(np.conj(nG) * sys.vpG)))
        E_alphaZ = sys.Ne * float(np.sum(alpha_z_ha(sys.Z, sys.rc, sys.ha_A))) / g.omega
    else:
        P_loc = (1.0 / 3.0) * float(np.real(np.sum(
            np.conj(nG) * sys.vG * (1.0 - g.G2 * sys.rc ** 2 / 2.0))))
        E_alphaZ = sys.Ne * float(np.sum(math.pi * sys.Z * sys.rc ** 2)) / g.omega
    P_ion = sys.E_ion / (3.0 * g.omega)
    return dict(F_tot=F_tot, F_el=F_el, F_s=F_s, minus_TS=-TS, E_H=E_H,
                E_loc=E_loc, F_xc=F_xc, E_ion=sys.E_ion, E_int=F_tot + TS,
                v=v, v_s=v_s, n=n, nG=nG, gradn=gradn, W=W,
                P=P_s + P_xc + P_H + P_loc + P_ion, P_s=P_s, P_xc=P_xc,
                P_H=P_H, P_loc=P_loc, P_ion=P_ion, E_alphaZ=E_alphaZ)


# ------------------------------------------- stress tensor (Eq. (StressTensor))
def stress(sys, ev):
    """Stress tensor Sigma_ab = (1/V) sum_nu (dF/dh_a,nu) h_b,nu of
    Eq. (StressTensor) at the density of `ev` (P = -Tr Sigma/3,
    Eq. (pressure)), term by term, under a homogeneous strain at fixed
    fractional coordinates and fixed V n(G):
      non-interacting  delta_ab/V int (f_s - n v_s) - (1/V) int W_a d_b n
                       (Eqs. (stressTF_a), (stressTF_b); W = d f_s/d grad n,
                       v_s the full functional derivative)
      XC               delta_ab/V int n (eps_xc - v_xc)   (Eq. (stressLSDAxc))
      Hartree          -delta_ab E_H/V + sum_G 4 pi |n(G)|^2 G_a G_b/G^4
      LPP              -delta_ab E_loc/V - 2 sum_G Re[n*(G) v'(G)] G_a G_b,
                       v' = dv/dG^2 at fixed V v(G) (Gaussian ion:
                       v (-rc^2/4 - 1/G^2); Eq. (E4A): from its dilation weights)
      ions             the Ewald stress (ewald_cell).
    Returns a dict of 3x3 arrays per term and their sum "Sigma"."""
    g = sys.grid
    V = g.omega
    I3 = np.eye(3)
    Gs = [np.broadcast_to(x, g.shape) for x in (g.Gx, g.Gy, g.Gz)]
    nG = ev["nG"]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv2 = np.where(g.G2 > 0.0, 1.0 / g.G2, 0.0)
    Ss = (ev["F_s"] - g.integrate(ev["n"] * ev["v_s"])) / V * I3
    if ev["W"] is not None:
        for a in range(3):
            for b in range(3):
                Ss[a, b] -= 0.5 / V * g.integrate(ev["W"][a] * ev["gradn"][b] + ev["W"][b] * ev["gradn"][a])
    Sxc = -ev["P_xc"] * I3
    hw = 4.0 * math.pi * np.abs(nG) ** 2 * inv2 * inv2
    SH = -ev["E_H"] / V * I3 + np.array([[np.sum(hw * Gs[a] * Gs[b]) for b in range(3)] for a in range(3)])
    if sys.lpp == "ha":
        dv = 1.5 * (sys.vpG - sys.vG) * inv2
    else:
        dv = sys.vG * (-sys.rc ** 2 / 4.0 - inv2)
    lw = np.real(np.conj(nG) * dv)
    Sloc = -ev["E_loc"] / V * I3 - 2.0 * np.array([[np.sum(lw * Gs[a] * Gs[b]) for b in range(3)]
                                                   for a in range(3)])
    cell = np.diag(g.L) if sys.cell is None else sys.cell
    Sion = ewald_cell(cell, sys.R, sys.Z)[2]
    tot = Ss + Sxc + SH + Sloc + Sion
    return dict(Sigma=tot, s=Ss, xc=Sxc, H=SH, loc=Sloc, ion=Sion)


# ---------------------------------------------------- minimisation (Sec. II)
def _mu_grad(sys, phi, v):
    """mu = int phi^2 v / int phi^2, g = 2 phi (v - mu), ||g|| = (dV sum g^2)^{1/2}."""
    mu = float(np.sum(phi * phi * v) / np.sum(phi * phi))
    gr = 2.0 * phi * (v - mu)
    return mu, gr, math.sqrt(sys.grid.dV * float(np.sum(gr * gr)))


def minimize(sys, phi0=None, gtol=1e-8, maxit=2000, theta0=0.05, ls_tol=0.1,
             max_ls=20, callback=None, e_tol=1e-11):
    """Direct minimisation of F_tot[n = phi^2] under int n = N_e (Sec. II).

    Nonlinear conjugate gradients; the paper names CG without details, so the
    scheme is a reading: Polak-Ribiere+ direction projected orthogonal to phi,
    restart along -g when not a descent direction, norm-preserving rotation
    phi(theta) = phi cos(theta) + dhat sin(theta) with ||dhat|| = ||phi||, and
    a line search on dE/dtheta (secant, regula falsi once bracketed) until
    |dE/dtheta| <= ls_tol |dE/dtheta(0)| at a point whose free energy lies
    below the sufficient-decrease line E(0) + 1e-4 theta dE/dtheta(0) (with
    a rounding allowance e_tol |E(0)|; a trial above it bounds the step).
    Stops when ||g|| < gtol.  Returns (phi, evaluation dict, stats dict).
    """
    g = sys.grid
    phi = (sys.uniform_phi() if phi0 is None else np.array(phi0, dtype=np.float64))
    phi *= math.sqrt(sys.Ne / g.integrate(phi * phi))     # dV sum phi^2 = N_e
    ev = evaluate(sys, phi)
    nevals = 1
    mu, gr, gnorm = _mu_grad(sys, phi, ev["v"])
    d_prev = gr_prev = None
    theta_prev = theta0
    it = 0
    status = "maxit"
    while it < maxit:
        if gnorm < gtol:
            status = "converged"
            break
        if gr_prev is None:
            d = -gr
        else:
            beta = max(0.0, float(np.sum(gr * (gr - gr_prev)) / np.sum(gr_prev * gr_prev)))
            d = -gr + beta * d_prev
        pp = float(np.sum(phi * phi))
        d = d - phi * (float(np.sum(phi * d)) / pp)
        if float(np.sum(d * gr)) >= 0.0:
            d = -gr
        dhat = d * math.sqrt(pp / float(np.sum(d * d)))
        D0 = g.dV * float(np.sum(2.0 * phi * ev["v"] * dhat))
        th, ev_new, phi_new, nls = _line_search(sys, phi, dhat, D0, theta_prev,
                                                ls_tol, max_ls, ev["F_tot"], e_tol)
        nevals += nls
        if th is None:
            if gr_prev is None:
                status = "linesearch"
                break
            d_prev = gr_prev = None          # restart along steepest descent
            continue
        theta_prev = th
        phi, ev = phi_new, ev_new
        gr_prev, d_prev = gr, d
        mu, gr, gnorm = _mu_grad(sys, phi, ev["v"])
        it += 1
        if callback is not None:
            callback(it, ev, gnorm)
    return phi, ev, dict(iterations=it, evaluations=nevals, gnorm=gnorm,
                         mu=mu, status=status)


def minimize_tn(sys, phi0=None, gtol=1e-8, maxit=500, inner_max=20, eta=0.1,
                fd_rel=1e-4, ls_tol=0.1, max_ls=20, e_tol=1e-11):
    """Truncated-Newton minimisation of F_tot[phi^2] under int n = N_e, the
    alternative to CG that PROFESS offers (Sec. II); the paper gives no
    details, so this is a reading.  Each outer step solves H d = -g on the
    tangent space (orthogonal to phi) by an inner CG truncated when
    ||r|| <= eta ||g||, after inner_max steps, or at non-positive curvature
    (then the last iterate, or -g at the first step).  H x is the central
    difference of the gradient map g(psi) = 2 psi (v[psi^2] - mu) along x,
    mu held at its current value, projected orthogonal to phi.  The step
    then takes the CG's norm-preserving rotation and line search, starting
    from the Newton angle ||d|| / ||phi||.  Returns (phi, ev, stats) with
    the evaluations spent on Hessian products counted in stats."""
    g = sys.grid
    phi = (sys.uniform_phi() if phi0 is None else np.array(phi0, dtype=np.float64))
    phi *= math.sqrt(sys.Ne / g.integrate(phi * phi))
    ev = evaluate(sys, phi)
    nevals, nhess = 1, 0
    mu, gr, gnorm = _mu_grad(sys, phi, ev["v"])
    it = 0
    status = "maxit"

    def proj(x):
        return x - phi * (float(np.sum(phi * x)) / float(np.sum(phi * phi)))

    while it < maxit:
        if gnorm < gtol:
            status = "converged"
            break
        b = -proj(gr)
        x = np.zeros_like(phi)
        r = b.copy()
        p = r.copy()
        rr = float(np.sum(r * r))
        bn = math.sqrt(float(np.sum(b * b)))
        for j in range(inner_max):
            h = fd_rel * math.sqrt(float(np.sum(phi * phi)) / float(np.sum(p * p)))
            gp = [2.0 * q * (evaluate(sys, q)["v"] - mu) for q in (phi + h * p, phi - h * p)]
            nevals += 2
            nhess += 1
            Hp = proj((gp[0] - gp[1]) / (2.0 * h))
            pHp = float(np.sum(p * Hp))
            if pHp <= 0.0:
                if j == 0:
                    x = b
                break
            a = rr / pHp
            x = x + a * p
            r = r - a * Hp
            rr_new = float(np.sum(r * r))
            if math.sqrt(rr_new) <= eta * bn:
                break
            p = r + (rr_new / rr) * p
            rr = rr_new
        d = proj(x)
        if float(np.sum(d * gr)) >= 0.0:
            d = b
        pp = float(np.sum(phi * phi))
        theta1 = min(math.sqrt(float(np.sum(d * d)) / pp), 1.0)
        dhat = d * math.sqrt(pp / float(np.sum(d * d)))
        D0 = g.dV * float(np.sum(2.0 * phi * ev["v"] * dhat))
        th, ev_new, phi_new, nls = _line_search(sys, phi, dhat, D0, theta1, ls_tol, max_ls,
                                                ev["F_tot"], e_tol)
        nevals += nls
        if th is None:
            status = "linesearch"
            break
        phi, ev = phi_new, ev_new
        mu, gr, gnorm = _mu_grad(sys, phi, ev["v"])
        it += 1
    return phi, ev, dict(iterations=it, evaluations=nevals, hessian_products=nhess,
                         gnorm=gnorm, mu=mu, status=status)


def _line_search(sys, phi, dhat, D0, theta1, ls_tol, max_ls, E0=None, e_tol=0.0):
    """Derivative line search in theta (reading of the CG step, Sec. II).

    Trial theta is accepted when |D| <= ls_tol |D0| and E(theta) <= E0 +
    1e-4 theta D0 + e_tol |E0|.  A trial above that line becomes the upper
    bracket whatever the sign of D there (the energy went up, so a minimum
    lies before it); with D <= 0 at that bracket the next trial bisects.
    """
    g = sys.grid
    lo, Dlo = 0.0, D0
    hi = Dhi = None
    hi_nod = False               # upper bracket from the energy test with D <= 0
    pa, Da = 0.0, D0            # last two points for the unbracketed secant
    th = theta1
    for k in range(max_ls):
        c, s = math.cos(th), math.sin(th)
        p = phi * c + dhat * s
        ev = evaluate(sys, p)
        D = g.dV * float(np.sum(2.0 * p * ev["v"] * (-phi * s + dhat * c)))
        up = (e_tol > 0.0 and E0 is not None
              and ev["F_tot"] > E0 + 1e-4 * th * D0 + e_tol * abs(E0))
        if not up and abs(D) <= ls_tol * abs(D0):
            return th, ev, p, k + 1
        if up:
            hi, Dhi, hi_nod = th, D, not (D > 0.0)
        elif D < 0.0:
            lo, Dlo = th, D
        else:
            hi, Dhi, hi_nod = th, D, False
        if hi is None:
            nxt = 4.0 * th
            if D > Da:
                sec = th - D * (th - pa) / (D - Da)
                nxt = min(sec, 4.0 * th)
            nxt = max(nxt, 1.1 * th)
            pa, Da = th, D
        elif hi_nod:
            nxt = 0.5 * (lo + hi)
        else:
            nxt = lo - Dlo * (hi - lo) / (Dhi - Dlo)
            w = hi - lo
            nxt = min(max(nxt, lo + 0.01 * w), hi - 0.01 * w)
        th = min(nxt, 1.5)
    if lo > 0.0:
        c, s = math.cos(lo), math.sin(lo)
        p = phi * c + dhat * s
        return lo, evaluate(sys, p), p, max_ls + 1
    return None, None, None, max_ls


# ------------------------------------------------ forces and pressure (Eq. M12)
def forces(sys, ev):
    """F_I = -int n grad_I v_ext - grad_I E_ion (Eq. (M12)).

    With the discrete v_ext = Re sum_G v(G) e^{iG.r}:
    F_I^loc = Omega Re sum_G i G w_I(G) e^{-iG.R_I} conj(n(G)), where
    w_I = Z_I w(G) for the Gaussian ion and Eq. (E4A)'s form for Heine-Abarenkov.
    """
    g = sys.grid
    F = np.zeros((len(sys.Z), 3))
    cn = np.conj(ev["nG"])
    for I in range(len(sys.Z)):
        if sys.lpp == "ha":
            wI = lpp_form_ha(g.G2, g.omega, sys.Z[I], sys.rc, sys.ha_A, sys.ha_qc)
        else:
            wI = sys.Z[I] * lpp_form(g.G2, g.omega, sys.rc)
        base = wI * structure_phase(g, sys.R[I]) * cn
        for a, Ga in enumerate((g.Gx, g.Gy, g.Gz)):
            F[I, a] = g.omega * float(np.real(np.sum(1j * Ga * base)))
    return F + sys.F_ion


# ------------------------------------------------------------ MD (Sec. V C)
class MDState:
    """Ion positions/velocities, a Nose-Hoover thermostat and the density
    history used for extrapolation."""

    def __init__(self, R, V, masses, T_ion_kelvin, dt_fs, tau_steps=100.0):
        self.R = np.array(R, dtype=np.float64)
        self.V = np.array(V, dtype=np.float64)
        self.m = np.array(masses, dtype=np.float64)
        self.dt = dt_fs * FS_AU
        self.kT = T_ion_kelvin * KB_HA_PER_K
        self.ndof = 3 * len(self.m) - 3
        tau = tau_steps * self.dt
        self.Q = self.ndof * self.kT * tau * tau / (4.0 * math.pi ** 2)
        self.xi = 0.0
        self.eta = 0.0
        self.phi = None
        self.phi_prev = None
        self.F = None
        self.ev = None

    def kinetic(self):
        return 0.5 * float(np.sum(self.m[:, None] * self.V * self.V))


def _nh_half(st):
    """Quarter-kick of xi, velocity scaling by exp(-xi dt/2), quarter-kick."""
    h = 0.5 * st.dt
    K = st.kinetic()
    st.xi += 0.5 * h * (2.0 * K - st.ndof * st.kT) / st.Q
    st.V *= math.exp(-st.xi * h)
    st.eta += st.xi * h
    K = st.kinetic()
    st.xi += 0.5 * h * (2.0 * K - st.ndof * st.kT) / st.Q


def md_prepare(sys, st, gtol=1e-8):
    """Minimise at the initial geometry and compute forces (step 0)."""
    sys.set_positions(st.R)
    phi, ev, stats = minimize(sys, None, gtol=gtol)
    st.phi, st.phi_prev, st.ev = phi, phi, ev
    st.F = forces(sys, ev)
    return stats


def md_step(sys, st, gtol=1e-8, thermostat=True):
    """One velocity-Verlet step with a Nose-Hoover thermostat (Trotter split).

    Readings (the paper's runs used QE's integrators, Fig. (P-QE)): density
    extrapolated as phi0 = normalise(2 phi_n - phi_{n-1}); COM velocity is
    not touched inside the step.
    """
    if thermostat:
        _nh_half(st)
    st.V += 0.5 * st.dt * st.F / st.m[:, None]
    st.R += st.dt * st.V
    sys.set_positions(st.R)
    guess = 2.0 * st.phi - st.phi_prev
    guess *= math.sqrt(sys.Ne / (sys.grid.dV * float(np.sum(guess * guess))))
    phi, ev, stats = minimize(sys, guess, gtol=gtol)
    st.phi_prev, st.phi, st.ev = st.phi, phi, ev
    st.F = forces(sys, ev)
    st.V += 0.5 * st.dt * st.F / st.m[:, None]
    if thermostat:
        _nh_half(st)
    return stats


def md_andersen(st, T_kelvin, prob, u, xi):
    """Andersen collisions (the thermostat of the paper's NVT runs, Sec. VI):
    ion I collides when u_I < prob and then takes a velocity drawn from the
    Maxwell-Boltzmann distribution at T, v_I = sqrt(kT/m_I) xi_I.  The
    uniform u[nat] and standard normal xi[nat,3] come in as inputs."""
    kT = T_kelvin * KB_HA_PER_K
    hit = np.asarray(u, dtype=np.float64) < prob
    xi = np.asarray(xi, dtype=np.float64).reshape(-1, 3)
    st.V[hit] = np.sqrt(kT / st.m[hit])[:, None] * xi[hit]
    return int(np.count_nonzero(hit))


def md_conserved(st):
    """Nose-Hoover extended energy K + F_tot + Q xi^2/2 + g kT eta."""
    return (st.kinetic() + st.ev["F_tot"] + 0.5 * st.Q * st.xi ** 2
            + st.ndof * st.kT * st.eta)
