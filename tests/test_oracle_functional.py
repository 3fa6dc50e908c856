"""Pins for the oracle's discrete functional, Hartree, pseudopotential, Ewald,
CG minimiser, forces (Eq. (M12)), pressure (Eq. (pressure)) and MD step.

Every check here is fixed by something other than the oracle's own formula:
finite differences of the discrete energy, closed-form lattice sums,
textbook Madelung constants, invariances, and limits.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import erf, erfc

import oracle as O
from paper_1406_0835_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def small_system(functional="fttf", grid=12, T=1.0e5, rc=0.25, xc=True):
    cfg = I.config_single_point()
    return O.System(cfg["L"], (grid, grid, grid), cfg["ions"], cfg["Z"], T,
                    functional, rc=rc, xc=xc)


@pytest.mark.parametrize("fn", ["fttf", "sga", "vt84f", "kst2", "apbef"])
def test_potential_is_derivative_of_discrete_energy(fn):
    s = small_system(fn)
    rng = np.random.default_rng(3)
    phi = s.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(s.grid.shape))
    ev = O.evaluate(s, phi)
    n = phi * phi
    for j in [(0, 0, 0), (3, 5, 7), (11, 2, 9), (6, 6, 6)]:
        h = 1e-4 * n[j]
        F = []
        for k in (-2, -1, 1, 2):
            nn = n.copy()
            nn[j] += k * h
            F.append(O.evaluate(s, np.sqrt(nn))["F_tot"])
        d = (F[0] - 8 * F[1] + 8 * F[2] - F[3]) / (12 * h) / s.grid.dV
        assert d == pytest.approx(ev["v"][j], rel=2e-8, abs=1e-9)


def test_gradient_and_divergence_are_adjoint():
    g = O.Grid((4.0, 5.0, 6.0), (12, 10, 8))
    rng = np.random.default_rng(1)
    n = rng.standard_normal(g.shape)
    W = rng.standard_normal((3,) + g.shape)
    lhs = np.sum(g.grad(n) * W)
    rhs = -np.sum(n * g.div(W))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_cosine_density_gradient_excess():
    """n = n0 (1 + eps cos Gx): F_SGA - F_TF = (1/144) h~(t0) n0 eps^2 G^2 Omega + O(eps^3),
    and VT84F's excess is that times (-mu + alpha + 5/3)/(5/27) (Eqs. (FGGA), (VT84F), (SGA-F))."""
    g = O.Grid((6.0, 6.0, 6.0), (24, 4, 4))
    n0, T, eps = 0.1, 0.3, 2e-3
    G = 2.0 * math.pi / 6.0
    x = np.arange(24) * 6.0 / 24
    n = n0 * (1.0 + eps * np.cos(G * x))[:, None, None] * np.ones(g.shape)
    gradn = g.grad(n)
    tf = g.integrate(O.fs_fttf(n, T)["f"])
    sga = g.integrate(O.fs_gga(n, gradn, T, O.FUNCTIONALS["sga"])["f"])
    vt = g.integrate(O.fs_gga(n, gradn, T, O.FUNCTIONALS["vt84f"])["f"])
    t0 = O.reduced_t(np.array([n0]), T)
    h0 = O.kappa_h(t0)[4][0]
    pred = h0 * n0 * eps ** 2 * G ** 2 * g.omega / 144.0
    assert sga - tf == pytest.approx(pred, rel=5e-3)
    c = -2.778 + 1.2965 + 5.0 / 3.0
    assert (vt - tf) / (sga - tf) == pytest.approx(c / (5.0 / 27.0), rel=5e-3)


def _ewald_real_self_bg(L, R, Z, a):
    """Real-space erfc lattice sum + self + background terms of the Ewald split."""
    L = np.asarray(L, float)
    omega = float(np.prod(L))
    E = 0.0
    nimg = [int(math.ceil(7.0 / a / L[k])) + 1 for k in range(3)]
    for I_ in range(len(Z)):
        for J in range(len(Z)):
            for i in range(-nimg[0], nimg[0] + 1):
                for j in range(-nimg[1], nimg[1] + 1):
                    for k in range(-nimg[2], nimg[2] + 1):
                        d = R[I_] - R[J] - np.array([i, j, k]) * L
                        r = math.sqrt(float(d @ d))
                        if r > 1e-12:
                            E += 0.5 * Z[I_] * Z[J] * erfc(a * r) / r
    E -= a / math.sqrt(math.pi) * float(np.sum(np.asarray(Z) ** 2))
    E -= math.pi * float(np.sum(Z)) ** 2 / (2.0 * omega * a * a)
    return E


def test_hartree_energy_of_periodic_gaussians():
    """Gaussian charges (alpha/pi)^{3/2} exp(-alpha r^2) in a neutralising background:
    E_H (Eq. (E2), G = 0 dropped) equals the reciprocal part of an Ewald sum with
    a^2 = alpha/2, i.e. E_Ewald - (real + self + background)(a)."""
    L = (5.0, 6.0, 7.0)
    g = O.Grid(L, (40, 48, 56))
    R = np.array([[1.0, 2.0, 3.0], [3.5, 1.0, 5.5]])
    Z = np.array([1.0, 2.0])
    alpha = 3.0
    xs = [np.arange(g.shape[k]) * L[k] / g.shape[k] for k in range(3)]
    X, Y, Zc = np.meshgrid(*xs, indexing="ij")
    n = np.zeros(g.shape)
    for I_ in range(2):
        for i in (-1, 0, 1):
            for j in (-1, 0, 1):
                for k in (-1, 0, 1):
                    d2 = ((X - R[I_, 0] - i * L[0]) ** 2 + (Y - R[I_, 1] - j * L[1]) ** 2
                          + (Zc - R[I_, 2] - k * L[2]) ** 2)
                    n += Z[I_] * (alpha / math.pi) ** 1.5 * np.exp(-alpha * d2)
    s = O.System(L, g.shape, R, Z, 1e4, "fttf")
    ev = O.evaluate(s, np.sqrt(n))
    a = math.sqrt(alpha / 2.0)
    E_total, _ = O.ewald(L, R, Z)
    ref = E_total - _ewald_real_self_bg(L, R, Z, a)
    assert ev["E_H"] == pytest.approx(ref, rel=1e-9)


def test_local_pseudopotential_real_space():
    """v_ext(G) = -4 pi Z exp(-G^2 rc^2/4)/(Omega G^2) is -Z erf(r/rc)/r (Sec. V A);
    with G = 0 dropped the periodic sum has zero mean.  Real-space reference:
    -Z [Ewald potential of a point charge] + Z sum_L erfc(r_L/rc)/r_L, mean removed."""
    L = (5.0, 5.5, 6.0)
    rc = 0.9                    # wide enough that v(G) has decayed at the grid's Nyquist
    g = O.Grid(L, (36, 40, 44))
    R = np.array([[1.2, 2.3, 3.1]])
    Z = np.array([1.0])
    vG = O.lpp_vG(g, R, Z, rc)
    v = g.to_r(vG)
    pts = [(0, 0, 0), (5, 17, 30), (20, 3, 11), (35, 39, 43)]
    a = 1.6
    omega = float(np.prod(L))
    km = 16
    K = np.array(np.meshgrid(*[np.arange(-km, km + 1)] * 3, indexing="ij")).reshape(3, -1).T
    Gv = 2 * math.pi * K / np.array(L)
    G2 = np.sum(Gv * Gv, axis=1)
    sel = G2 > 0
    Gv, G2 = Gv[sel], G2[sel]
    ref = []
    for p in pts:
        r = np.array([p[k] * L[k] / g.shape[k] for k in range(3)])
        phiE = 0.0
        scr = 0.0
        for i in range(-4, 5):
            for j in range(-4, 5):
                for k in range(-4, 5):
                    d = r - R[0] - np.array([i, j, k]) * np.array(L)
                    rr = math.sqrt(float(d @ d))
                    phiE += erfc(a * rr) / rr
                    scr += erfc(rr / rc) / rr
        phiE += (4 * math.pi / omega) * float(np.sum(np.exp(-G2 / (4 * a * a)) / G2
                                                     * np.cos(Gv @ (r - R[0]))))
        phiE -= math.pi / (omega * a * a)
        ref.append(-Z[0] * phiE + Z[0] * scr)
    # the grid function has zero mean; the lattice sum's mean is -pi Z rc^2/Omega
    # (the G -> 0 limit of v(G) + 4 pi Z/(Omega G^2))
    ref = np.array(ref) - math.pi * Z[0] * rc * rc / omega
    got = np.array([v[p] for p in pts])
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-11)


def test_ewald_madelung_and_invariances():
    gold = json.load(open(os.path.join(GOLD, "madelung.json")))
    E, F = O.ewald([1.0, 1.0, 1.0], [[0.1, 0.2, 0.3]], [1.0])
    assert E == pytest.approx(gold["sc_energy_per_ion_times_a"], rel=1e-11)
    Lb = 2.0
    E, F = O.ewald([Lb] * 3, [[0, 0, 0], [1.0, 1.0, 1.0]], [1.0, 1.0])
    rws = (3 * Lb ** 3 / (2 * 4 * math.pi)) ** (1 / 3)
    assert E / 2 * rws == pytest.approx(gold["bcc_energy_per_ion_times_rws"], rel=1e-11)
    assert np.max(np.abs(F)) < 1e-12                 # perfect lattice: no force
    L = [3.0, 4.0, 5.0]
    R = np.array([[0.1, 0.2, 0.3], [1.5, 2.1, 3.3], [2.9, 0.1, 4.0]])
    Z = [1.0, 2.0, 1.0]
    Es = [O.ewald(L, R, Z, alpha=a)[0] for a in (0.6, 1.3, 3.0)]
    assert max(Es) - min(Es) < 1e-13 * abs(Es[0])   # splitting independence
    E, F = O.ewald(L, R, Z)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-12     # Newton's third law
    h = 1e-5
    for I_ in range(3):
        for a in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[I_, a] += h
            Rm[I_, a] -= h
            fd = -(O.ewald(L, Rp, Z)[0] - O.ewald(L, Rm, Z)[0]) / (2 * h)
            assert fd == pytest.approx(F[I_, a], abs=1e-8)


def test_minimiser_constraint_and_euler_equation():
    s = small_system("sga", grid=12)
    phi, ev, st = O.minimize(s, gtol=1e-9)
    assert st["status"] == "converged"
    assert s.grid.integrate(phi * phi) == pytest.approx(s.Ne, rel=1e-13)
    # Euler equation (E10): v - mu vanishes where the density is
    resid = np.abs(ev["v"] - st["mu"]) * phi
    assert np.max(resid) < 1e-8
    # a minimum: random norm-preserving rotations raise F
    rng = np.random.default_rng(4)
    for _ in range(3):
        d = rng.standard_normal(phi.shape)
        d -= phi * np.sum(phi * d) / np.sum(phi * phi)
        d *= math.sqrt(np.sum(phi * phi) / np.sum(d * d))
        for th in (1e-3, -1e-3):
            p = phi * math.cos(th) + d * math.sin(th)
            assert O.evaluate(s, p)["F_tot"] > ev["F_tot"]


@pytest.mark.parametrize("fn", ["fttf", "vt84f"])
def test_forces_are_derivatives_of_minimised_energy(fn):
    """Eq. (M12): at electronic equilibrium F_I = -dF_tot/dR_I."""
    s = small_system(fn, grid=12)
    phi, ev, _ = O.minimize(s, gtol=1e-11)
    F = O.forces(s, ev)
    R0 = s.R.copy()
    h = 2e-4
    for I_, a in ((0, 0), (3, 2)):
        E = []
        for k in (-1, 1):
            R = R0.copy()
            R[I_, a] += k * h
            s.set_positions(R)
            E.append(O.minimize(s, phi, gtol=1e-11)[1]["F_tot"])
        s.set_positions(R0)
        fd = -(E[1] - E[0]) / (2 * h)
        assert fd == pytest.approx(F[I_, a], rel=1e-5, abs=1e-7)


def test_net_force_vanishes_on_a_resolving_grid():
    """Translation invariance: sum_I F_I = 0 once the grid resolves the
    pseudopotential (rc = 0.8 bohr, 16^3); coarse grids add an egg-box force."""
    s = small_system("sga", grid=16, rc=0.8)
    phi, ev, _ = O.minimize(s, gtol=1e-10)
    F = O.forces(s, ev)
    assert np.max(np.abs(F.sum(axis=0))) < 1e-7 * np.max(np.abs(F))


@pytest.mark.parametrize("fn", ["fttf", "sga"])
def test_pressure_is_volume_derivative(fn):
    """Eq. (pressure): P = -dF_tot/dOmega with fractional coordinates and the
    grid count fixed, at the minimised density of each volume."""
    cfg = I.config_single_point()
    L0 = np.array(cfg["L"])
    frac = cfg["ions"] / L0

    def F_at(lam, phi0=None):
        L = L0 * lam
        s = O.System(L, (12, 12, 12), frac * L, cfg["Z"], 1e5, fn)
        phi, ev, _ = O.minimize(s, phi0, gtol=1e-11)
        return s, phi, ev

    s, phi, ev = F_at(1.0)
    d = 1e-4
    Fp = F_at(1.0 + d, phi)[2]["F_tot"]
    Fm = F_at(1.0 - d, phi)[2]["F_tot"]
    omega = s.grid.omega
    dFdOmega = (Fp - Fm) / (omega * ((1 + d) ** 3 - (1 - d) ** 3))
    assert ev["P"] == pytest.approx(-dFdOmega, rel=2e-6)


def test_translation_by_grid_vector():
    s = small_system("sga", grid=12)
    phi, ev, _ = O.minimize(s, gtol=1e-10)
    h = s.grid.L[0] / 12
    R = s.R.copy()
    R[:, 0] += 2 * h
    s2 = small_system("sga", grid=12)
    s2.set_positions(R)
    phi2, ev2, _ = O.minimize(s2, gtol=1e-10)
    np.testing.assert_allclose(ev2["n"], np.roll(ev["n"], 2, axis=0), rtol=1e-7, atol=1e-10)
    assert ev2["F_tot"] == pytest.approx(ev["F_tot"], rel=1e-12)
    np.testing.assert_allclose(O.forces(s2, ev2), O.forces(s, ev), atol=1e-8)


def test_md_time_reversible_and_second_order():
    cfg = I.config_single_point()
    s = O.System(cfg["L"], (12, 12, 12), cfg["ions"], cfg["Z"], 1e5, "fttf", rc=0.6)
    V = I.maxwell_boltzmann(8, 1e5, seed=3)
    masses = np.full(8, I.M_H_AMU * I.AMU_ME)
    st = O.MDState(cfg["ions"], V, masses, 1e5, dt_fs=0.2)
    O.md_prepare(s, st, gtol=1e-11)
    R0 = st.R.copy()
    for _ in range(3):
        O.md_step(s, st, gtol=1e-11, thermostat=False)
    st.V = -st.V
    st.phi_prev = st.phi                    # restart extrapolation on reversal
    for _ in range(3):
        O.md_step(s, st, gtol=1e-11, thermostat=False)
    assert np.max(np.abs(st.R - R0)) < 1e-7
    # Nose-Hoover extended energy: velocity Verlet + Trotter split is second
    # order, so halving dt over the same time span cuts its error about 4x
    dev = []
    for dt, nsteps in ((0.1, 4), (0.05, 8)):
        st = O.MDState(cfg["ions"], V, masses, 1e5, dt_fs=dt)
        O.md_prepare(s, st, gtol=1e-11)
        H0 = O.md_conserved(st)
        d = 0.0
        for _ in range(nsteps):
            O.md_step(s, st, gtol=1e-11)
            d = max(d, abs(O.md_conserved(st) - H0))
        dev.append(d)
    assert 2.5 < dev[0] / dev[1] < 6.0


def test_andersen_collisions():
    """Andersen thermostat (the paper's NVT runs, Sec. VI): exactly the ions
    with u < prob are redrawn, from Maxwell-Boltzmann at T (equipartition:
    mean kinetic energy 3 kT/2 per ion, per-component variance kT/m)."""
    n = 20000
    masses = np.where(np.arange(n) % 2 == 0, 1.0, 4.0) * I.M_H_AMU * I.AMU_ME
    V0 = np.full((n, 3), 1e-3)
    st = O.MDState(np.zeros((n, 3)), V0, masses, 1e5, dt_fs=0.2)
    u, xi = I.andersen_draws(n, seed=5)
    assert O.md_andersen(st, 1e5, 0.0, u, xi) == 0
    assert np.array_equal(st.V, V0)
    hit = O.md_andersen(st, 1e5, 0.3, u, xi)
    changed = np.any(st.V != V0, axis=1)
    assert hit == np.count_nonzero(u < 0.3) and np.array_equal(changed, u < 0.3)
    assert abs(hit / n - 0.3) < 0.02
    O.md_andersen(st, 1e5, 1.0, u, xi)
    kT = 1e5 * O.KB_HA_PER_K
    K = 0.5 * np.sum(masses[:, None] * st.V ** 2, axis=1)
    # sampling error of the mean of (kT/2) chi^2_3 over n ions: 0.82 kT/sqrt(n)
    assert abs(np.mean(K) / (1.5 * kT) - 1.0) < 4 * 0.816 / math.sqrt(n)
    for sel in (slice(0, None, 2), slice(1, None, 2)):
        var = np.var(st.V[sel]) * masses[sel][0] / kT
        assert abs(var - 1.0) < 0.03


@pytest.mark.parametrize("fn", ["fttf", "sga"])
def test_truncated_newton_reaches_the_cg_minimum(fn):
    """The truncated-Newton alternative (Sec. II) stops at the same
    constrained minimum as the CG: one density, one free energy."""
    s = small_system(fn)
    p1, e1, s1 = O.minimize(s, gtol=1e-9)
    p2, e2, s2 = O.minimize_tn(s, gtol=1e-9)
    assert s2["status"] == "converged" and s2["gnorm"] < 1e-9
    assert e2["F_tot"] == pytest.approx(e1["F_tot"], rel=1e-12)
    assert np.max(np.abs(e2["n"] - e1["n"])) < 1e-8 * np.max(e1["n"])
    assert abs(s.grid.integrate(e2["n"]) - s.Ne) < 1e-12 * s.Ne
    assert s2["iterations"] < s1["iterations"]       # Newton steps: fewer, dearer
