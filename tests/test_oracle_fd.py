"""Pins for the oracle's Fermi-Dirac integrals and kappa(t), h~(t).

Each pin is fixed by mathematics independent of the oracle's quadrature:
closed forms at eta = 0, the classical series, the Sommerfeld limits, the
ideal-gas identities behind Eqs. (tred), (fTF), (vTF), (stressTF_a), central
finite differences, and the finite-T Lindhard response for h~.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O

NU = (-0.5, 0.5, 1.5)


def eta_dirichlet(s):
    """Dirichlet eta: F_j(0) = eta_D(j+1) = (1 - 2^{-j}) zeta(j+1)."""
    return (1.0 - 2.0 ** (1.0 - s)) * special.zeta(s)


def test_moments_at_zero_closed_form():
    m = O.fd_moments(np.array([0.0]))[0]
    # I_nu(0) = Gamma(nu+1) F_nu(0); d^k I_{-1/2}/deta^k = Gamma(1/2) F_{-1/2-k}
    want = [special.gamma(nu + 1.0) * eta_dirichlet(nu + 1.0) for nu in NU]
    want += [math.sqrt(math.pi) * eta_dirichlet(0.5 - k) for k in (1, 2, 3)]
    for got, ref in zip(m, want):
        assert got == pytest.approx(ref, rel=5e-14, abs=1e-15)


@pytest.mark.parametrize("eta", [-40.0, -12.0, -4.0, -2.0])
def test_moments_classical_series(eta):
    # 1/(1+e^{x-eta}) = sum_k (-1)^{k+1} e^{k(eta-x)} for eta < x gives
    # I_nu = Gamma(nu+1) sum_k (-1)^{k+1} e^{k eta} / k^{nu+1}.
    k = np.arange(1, 200, dtype=np.float64)
    sgn = (-1.0) ** (k + 1)
    ek = np.exp(k * eta)
    want = [special.gamma(nu + 1.0) * np.sum(sgn * ek / k ** (nu + 1.0)) for nu in NU]
    want += [math.sqrt(math.pi) * np.sum(sgn * ek * k ** p / k ** 0.5) for p in (1, 2, 3)]
    m = O.fd_moments(np.array([eta]))[0]
    for got, ref in zip(m, want):
        assert got == pytest.approx(ref, rel=2e-14)


@pytest.mark.parametrize("eta", [45.0, 300.0, 1.0e4])
def test_moments_degenerate_leading_terms(eta):
    # Sommerfeld: I_nu = eta^{nu+1}/(nu+1) [1 + (pi^2/6)(nu+1)nu eta^{-2} + ...]
    m = O.fd_moments(np.array([eta]))[0]
    for got, nu in zip(m[:3], NU):
        lead = eta ** (nu + 1.0) / (nu + 1.0) * (1.0 + math.pi ** 2 / 6.0 * (nu + 1.0) * nu / eta ** 2)
        assert got == pytest.approx(lead, rel=10.0 / eta ** 4)
    # derivatives of I_{-1/2} = 2 eta^{1/2}(1 - pi^2/(24 eta^2))
    d1 = eta ** -0.5 * (1.0 + math.pi ** 2 / 8.0 / eta ** 2)
    d2 = -0.5 * eta ** -1.5 * (1.0 + 5.0 * math.pi ** 2 / 8.0 / eta ** 2)
    assert m[3] == pytest.approx(d1, rel=30.0 / eta ** 4)
    assert m[4] == pytest.approx(d2, rel=300.0 / eta ** 4)


def test_quadrature_and_series_join_at_40():
    # quadrature just below eta = 40, Sommerfeld series at 40; first-order
    # Taylor step with the derivatives dI_{1/2} = I_{-1/2}/2, dI_{3/2} = (3/2) I_{1/2}
    de = 1e-9
    lo = O.fd_moments(np.array([40.0 - de]))[0]
    hi = O.fd_moments(np.array([40.0]))[0]
    slope = np.array([hi[3], 0.5 * hi[0], 1.5 * hi[1], hi[4], hi[5]])
    np.testing.assert_allclose(lo[:4] + de * slope[:4], hi[:4], rtol=1e-13)
    np.testing.assert_allclose(lo[4] + de * slope[4], hi[4], rtol=1e-11)


def test_moments_against_independent_quadrature():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for eta in (-3.0, 0.7, 12.0, 39.0, 150.0):
        e = mp.mpf(eta)
        f = lambda x: 1 / (1 + mp.e ** (x - e))
        pts = sorted(set([0, max(e - 30, 0), max(e, 0), max(e, 0) + 15, max(e, 0) + 90]))
        ref = [mp.quad(lambda x: x ** nu * f(x), pts) for nu in NU]
        ref.append(mp.quad(lambda x: x ** -0.5 * f(x) * (1 - f(x)), pts))
        m = O.fd_moments(np.array([eta]))[0]
        for got, r in zip(m[:4], ref):
            assert got == pytest.approx(float(r), rel=1e-13)


def test_eta_inversion():
    t = np.logspace(-5, 6, 57)
    eta = O.eta_of_t(t)
    m = O.fd_moments(eta)
    np.testing.assert_allclose(m[:, 1], (2.0 / 3.0) * t ** -1.5, rtol=1e-14)


def test_kappa_limits():
    t = np.array([1e-4, 3e-4])
    _, kap, dk, d2k, h, dh, d2h = O.kappa_h(t)
    # T -> 0 Sommerfeld: kappa = 1 - (5 pi^2/12) t^2, h~ = 1 + (pi^2/3) t^2
    np.testing.assert_allclose(kap, 1.0 - 5.0 * math.pi ** 2 / 12.0 * t ** 2, rtol=1e-12)
    np.testing.assert_allclose(dk, -5.0 * math.pi ** 2 / 6.0 * t, rtol=1e-5)
    np.testing.assert_allclose(h, 1.0 + math.pi ** 2 / 3.0 * t ** 2, rtol=1e-12)
    np.testing.assert_allclose(dh, 2.0 * math.pi ** 2 / 3.0 * t, rtol=1e-5)
    z = O.xi_zeta(t)
    np.testing.assert_allclose(z["zeta"], 5.0 * math.pi ** 2 / 6.0 * t ** 2, rtol=1e-5)
    # high T, classical ideal gas: kappa = (5/3) t [eta - 1] with
    # e^eta = (4/(3 sqrt(pi))) t^{-3/2}, first quantum correction in z = e^eta:
    # I_{1/2}/Gamma(3/2) = z - z^2/2^{3/2}, I_{3/2}/Gamma(5/2) = z - z^2/2^{5/2}
    t = np.array([1e3, 1e5])
    y = (2.0 / 3.0) * t ** -1.5
    zz = y / special.gamma(1.5)
    zz = zz + zz ** 2 / 2 ** 1.5 + zz ** 3 * (0.25 - 1.0 / 3 ** 1.5)   # series inversion
    eta = np.log(zz)
    I32 = special.gamma(2.5) * (zz - zz ** 2 / 2 ** 2.5 + zz ** 3 / 3 ** 2.5)
    kref = (5.0 / 3.0) * t * (eta - (2.0 / 3.0) * I32 / y)
    _, kap, _, _, h, _, _ = O.kappa_h(t)
    np.testing.assert_allclose(kap, kref, rtol=1e-13)
    np.testing.assert_allclose(h, 3.0, rtol=1e-3)
    z = O.xi_zeta(t)
    np.testing.assert_allclose(z["xi"], 2.5 * t, rtol=1e-4)   # tau0 xi -> (3/2) n T


@pytest.mark.parametrize("t0,rtol", [(2e-3, 1e-6), (0.05, 2e-9), (0.3, 2e-9), (1.0, 2e-9),
                                     (4.0, 2e-9), (60.0, 2e-9), (3e3, 2e-9)])
def test_t_derivatives_by_finite_differences(t0, rtol):
    # at t = 2e-3 the FD quotient is limited by the cancellation inside
    # kappa' = (5/3)[eta - (5/3) I_{3/2}/y] with eta ~ 500
    hstep = 1e-3 * t0
    ts = t0 + hstep * np.array([-2.0, -1.0, 1.0, 2.0])
    out = np.array(O.kappa_h(ts))
    c = np.array(O.kappa_h(np.array([t0])))[:, 0]
    fd = (out[:, 0] - 8 * out[:, 1] + 8 * out[:, 2] - out[:, 3]) / (12 * hstep)
    # dkappa, d2kappa, dh, d2h against FD of kappa, dkappa, h, dh
    pairs = ((1, 2), (2, 3), (4, 5), (5, 6))
    if t0 > 100.0:
        pairs = pairs[:2]    # h~ - 3 ~ t^{-3/2} there: its FD quotients are rounding noise
    for val_idx, der_idx in pairs:
        scale = max(abs(c[der_idx]), 1e-6 * max(abs(c[val_idx]), 1.0) / t0)
        assert abs(fd[val_idx] - c[der_idx]) <= rtol * scale + 1e-12 * abs(c[val_idx]) / t0


@pytest.mark.parametrize("T,n", [(0.3, 0.09), (0.03, 0.35), (12.0, 0.35), (0.01, 5.0)])
def test_uniform_gas_identities(T, n):
    """ftTF potential of a uniform gas is the ideal-gas chemical potential T eta,
    and n v - f is its pressure (2 sqrt2/(3 pi^2)) T^{5/2} I_{3/2} (Eqs. (vTF), (stressTF_a))."""
    n = np.array([n])
    fs = O.fs_fttf(n, T)
    t = O.reduced_t(n, T)
    eta = O.eta_of_t(t)
    m = O.fd_moments(eta)[0]
    assert fs["dfdn"][0] == pytest.approx(T * eta[0], rel=1e-12, abs=1e-13)
    P = 2.0 * math.sqrt(2.0) / (3.0 * math.pi ** 2) * T ** 2.5 * m[2]
    assert (n * fs["dfdn"] - fs["f"])[0] == pytest.approx(P, rel=1e-12)
    # density consistency: n = (sqrt2/pi^2) T^{3/2} I_{1/2}(eta)
    assert math.sqrt(2.0) / math.pi ** 2 * T ** 1.5 * m[1] == pytest.approx(n[0], rel=1e-13)
    # kinetic part is (3/2) P; entropic part T s = (5/2) P - n T eta
    assert fs["f_kin"][0] == pytest.approx(1.5 * P, rel=1e-12)
    assert fs["f_ent"][0] == pytest.approx(2.5 * P - n[0] * T * eta[0], rel=1e-9, abs=1e-14)


def _lindhard_h(eta):
    """h~ from the finite-T Lindhard function (Maldague average of the T = 0
    response over -df/dmu'), as 36 n b with -1/chi(q) = a + b q^2 + ..."""
    T = 1.0
    mu = eta * T

    def chi(q):
        def integrand(mp_):
            kf = math.sqrt(2.0 * mp_)
            z = q / (2.0 * kf)
            if z < 1e-3:
                F = 1.0 - z * z / 3.0 - z ** 4 / 15.0 - z ** 6 / 35.0
            else:
                F = 0.5 + (1.0 - z * z) / (4.0 * z) * math.log(abs((1.0 + z) / (1.0 - z)))
            x = (mp_ - mu) / T
            w = 1.0 / (4.0 * T * math.cosh(0.5 * x) ** 2)
            return -(kf / math.pi ** 2) * F * w
        hi = max(mu, 0.0) + 60.0 * T
        pts = [p for p in (q * q / 8.0, mu) if 0.0 < p < hi]
        val, _ = integrate.quad(integrand, 0.0, hi, points=pts or None,
                                epsabs=0.0, epsrel=1e-13, limit=400)
        return val
    c0 = -1.0 / chi(0.0)
    qs = np.array([0.05, 0.1, 0.2]) * math.sqrt(max(mu, 0.0) + T)
    bq = np.array([(-1.0 / chi(q) - c0) / q ** 2 for q in qs])
    # b(q) = b + d q^2 + e q^4: solve for b
    A = np.vstack([np.ones(3), qs ** 2, qs ** 4]).T
    b = np.linalg.solve(A, bq)[0]
    m = O.fd_moments(np.array([eta]))[0]
    n = math.sqrt(2.0) / math.pi ** 2 * T ** 1.5 * m[1]
    return 36.0 * n * b


@pytest.mark.parametrize("eta", [-2.0, 0.5, 3.0, 12.0])
def test_htilde_is_the_lindhard_gradient_coefficient(eta):
    t = (1.5 * O.fd_moments(np.array([eta]))[0][1]) ** (-2.0 / 3.0)
    h = O.kappa_h(np.array([t]))[4][0]
    assert h == pytest.approx(_lindhard_h(eta), rel=1e-6)


def test_sga_assembly_collapses_to_gradient_corrected_tf():
    """Eqs. (FGGA), (s_s), (SGA-F): SGA = tau0 kappa + (1/72) h~ |grad n|^2 / n."""
    rng = np.random.default_rng(7)
    n = np.exp(rng.uniform(-5, 2, 200))
    gradn = rng.standard_normal((3, 200)) * n
    T = 0.2
    fs = O.fs_gga(n, gradn, T, O.FUNCTIONALS["sga"])
    t = O.reduced_t(n, T)
    _, kap, _, _, h, _, _ = O.kappa_h(t)
    ref = O.C_TF * n ** (5.0 / 3.0) * kap + h / 72.0 * np.sum(gradn ** 2, axis=0) / n
    np.testing.assert_allclose(fs["f"], ref, rtol=1e-12)
    # with F = 1 the generic form is finite-T TF
    one = lambda x: (np.ones_like(x), np.zeros_like(x))
    fs1 = O.fs_gga(n, gradn, T, one)
    np.testing.assert_allclose(fs1["f"], O.fs_fttf(n, T)["f"], rtol=1e-13)
    np.testing.assert_allclose(fs1["dfdn"], O.fs_fttf(n, T)["dfdn"], rtol=1e-11, atol=1e-14)


def test_enhancement_factors_match_printed_constants():
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    x = np.array([1e-12, 0.3, 2.0])
    v = gold["vt84f"]
    F, dF = O.F_vt84f(x, mu=v["mu"], alpha=v["alpha"])
    Fo, dFo = O.FUNCTIONALS["vt84f"](x)
    np.testing.assert_array_equal(F, Fo)
    # small-s coefficient -mu + alpha + 5/3 ~ 5/27 (the SGA value)
    assert dFo[0] == pytest.approx(-v["mu"] + v["alpha"] + 5.0 / 3.0, rel=1e-7)
    assert abs(dFo[0] - gold["sga"]["mu"]) < 2e-5
    for name in ("kst2", "tw"):
        g = gold[name]
        F, _ = O.FUNCTIONALS[name](x)
        np.testing.assert_allclose(F, 1 + g["C1"] * x / (1 + g["a1"] * x), rtol=1e-15)
    g = gold["apbef"]
    F, _ = O.FUNCTIONALS["apbef"](x)
    np.testing.assert_allclose(F, 1 + g["C1"] * x / (1 + g["C1"] / g["a1_over"] * x), rtol=1e-15)
    for name in ("sga", "vwtf"):
        F, _ = O.FUNCTIONALS[name](x)
        np.testing.assert_allclose(F, 1 + gold[name]["mu"] * x, rtol=1e-15)
    assert O.C_TF == pytest.approx(gold["c_tf_formula"]["value"], rel=1e-15)
    # derivatives of the enhancement factors against FD
    for name in ("vt84f", "kst2", "sga"):
        for x0 in (1e-3, 0.4, 3.0):
            hs = 1e-5 * x0
            Fp = O.FUNCTIONALS[name](np.array([x0 + hs]))[0][0]
            Fm = O.FUNCTIONALS[name](np.array([x0 - hs]))[0][0]
            d = O.FUNCTIONALS[name](np.array([x0]))[1][0]
            assert (Fp - Fm) / (2 * hs) == pytest.approx(d, rel=1e-7, abs=1e-9)


def test_pz81_branches_meet_at_rs_1():
    """The two PZ81 correlation branches meet with equal eps_c and v_c at
    r_s = 1, and the derived C, D round to the published 0.0020, -0.0116."""
    assert round(O.PZ["C"], 4) == 0.0020 and round(O.PZ["D"], 4) == -0.0116
    n1 = 3.0 / (4.0 * math.pi)                       # r_s = 1
    e_lo, v_lo = O.pz81(np.array([n1 * (1 + 1e-12)]))  # r_s just below 1: log branch
    e_hi, v_hi = O.pz81(np.array([n1 * (1 - 1e-12)]))  # just above: Pade branch
    assert abs(e_lo[0] - e_hi[0]) < 1e-12 and abs(v_lo[0] - v_hi[0]) < 1e-11
    # Pade value at r_s = 1 plus exchange, written out
    ex = -0.4581652932831429
    assert e_hi[0] == pytest.approx(ex - 0.1423 / (1 + 1.0529 + 0.3334), abs=1e-12)


def test_pz81_exchange_and_potential():
    n = np.array([1e-3, 0.05, 0.0885, 0.2387, 0.4, 3.0])
    eps, v = O.pz81(n)
    rs = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    ex = -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * n ** (1.0 / 3.0)
    # exchange alone is -(3/4)(3/pi)^{1/3} n^{1/3} = -0.4581652932831429 / r_s
    np.testing.assert_allclose(ex, -0.4581652932831429 / rs, rtol=1e-14)
    # v_xc = d(n eps)/dn by central differences
    hs = 1e-6 * n
    ep, _ = O.pz81(n + hs)
    em, _ = O.pz81(n - hs)
    fd = ((n + hs) * ep - (n - hs) * em) / (2 * hs)
    np.testing.assert_allclose(v, fd, rtol=1e-8)
