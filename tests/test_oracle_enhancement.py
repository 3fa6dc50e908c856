"""Pins of the oracle's enhancement factors (Sec. III B, Eqs. (VT84F),
(KST2F), (SGA-F)) away from small s.

Each factor is written out again here in the paper's own variable s (not
the oracle's x = s^2), evaluated in mpmath at 30 digits term by term, and
differentiated numerically by mpmath; the oracle's F(x) and dF/dx must agree
to binary64 rounding.  A slip in any one term of the oracle (a sign, an
exponent m/2 or n/2, a constant) moves F at moderate s by far more than the
tolerance.  VT84F also has a closed large-s limit: the (1 - e^{-alpha s^4})
factor tends to 1, so F - (5/3) s^2 -> s^{-2}.
"""
import mpmath as mp
import numpy as np
import pytest

import oracle as O

mp.mp.dps = 30

VT_MU, VT_ALPHA, VT_M, VT_N = mp.mpf("2.778"), mp.mpf("1.2965"), 8, 4


def vt84f_s(s):
    """Eq. (VT84F): 1 - mu s^2 e^{-alpha s^2}/(1 + mu s^2)
    + (1 - e^{-alpha s^{m/2}}) (s^{-n/2} - 1) + (5/3) s^2, m = 8, n = 4."""
    s = mp.mpf(s)
    t1 = VT_MU * s ** 2 * mp.exp(-VT_ALPHA * s ** 2) / (1 + VT_MU * s ** 2)
    t2 = (1 - mp.exp(-VT_ALPHA * s ** (VT_M // 2))) * (s ** (-(VT_N // 2)) - 1)
    t3 = mp.mpf(5) / 3 * s ** 2
    return 1 - t1 + t2 + t3


def kst2_s(C1, a1):
    """Eq. (KST2F): 1 + C1 s^2/(1 + a1 s^2)."""
    C1, a1 = mp.mpf(C1), mp.mpf(a1)
    return lambda s: 1 + C1 * mp.mpf(s) ** 2 / (1 + a1 * mp.mpf(s) ** 2)


def sga_s(mu):
    """Eq. (SGA-F): 1 + mu s^2."""
    mu = mp.mpf(mu)
    return lambda s: 1 + mu * mp.mpf(s) ** 2


CASES = {
    "vt84f": vt84f_s,
    "kst2": kst2_s("2.03087", "0.29424"),
    "tw": kst2_s("0.2319", "0.2748"),
    "apbef": kst2_s("0.23889", mp.mpf("0.23889") / mp.mpf("0.804")),
    "sga": sga_s(mp.mpf(5) / 27),
    "vwtf": sga_s(mp.mpf(5) / 3),
}

XS = [0.05, 0.3, 0.5, 1.0, 2.0, 3.7, 8.0, 20.0]


@pytest.mark.parametrize("fn", sorted(CASES))
def test_enhancement_factor_and_derivative_against_mpmath(fn):
    Fs = CASES[fn]
    F, dF = O.FUNCTIONALS[fn](np.array(XS))
    for k, x in enumerate(XS):
        s = mp.sqrt(mp.mpf(x))
        ref = Fs(s)
        # dF/dx = (dF/ds) / (2 s), the derivative taken by mpmath
        dref = mp.diff(Fs, s) / (2 * s)
        assert abs(F[k] - float(ref)) <= 4e-16 * max(1.0, abs(float(ref))), (fn, x, F[k], ref)
        assert abs(dF[k] - float(dref)) <= 1e-14 * max(1.0, abs(float(dref))), (fn, x, dF[k], dref)


def test_vt84f_printed_points():
    """Values at x = s^2 in {0.5, 2, 8} from the 30-digit evaluation (the
    terms at those points: at x = 8 the Gaussian factor is 1 to 36 digits
    and the first term is 2e-5, so F = 1 - 2.0e-5 + (1/8 - 1) + 40/3)."""
    F, _ = O.F_vt84f(np.array([0.5, 2.0, 8.0]))
    for x, got in zip((0.5, 2.0, 8.0), F):
        assert abs(got - float(vt84f_s(mp.sqrt(x)))) <= 4e-16 * abs(got)
    e8 = float(VT_MU * 8 * mp.exp(-VT_ALPHA * 8) / (1 + VT_MU * 8))
    assert abs(F[2] - (1.0 - e8 + (1.0 / 8.0 - 1.0) + 40.0 / 3.0)) < 1e-14 * F[2]


@pytest.mark.parametrize("x", [30.0, 100.0, 1.0e4])
def test_vt84f_large_s_limit(x):
    """F - (5/3) x -> 1/x (the first term decays as e^{-alpha x})."""
    F, dF = O.F_vt84f(np.array([x]))
    tail = float(VT_MU * x * mp.exp(-VT_ALPHA * x) / (1 + VT_MU * x))
    assert abs((F[0] - 5.0 * x / 3.0) - (1.0 / x - tail)) <= 1e-15 * F[0]
    assert abs(dF[0] - (5.0 / 3.0 - 1.0 / x ** 2)) <= 1e-12


def test_vt84f_small_s_limit_and_continuity():
    """At x -> 0 the oracle's removable-singularity branch joins the formula."""
    F0, dF0 = O.F_vt84f(np.array([0.0]))
    F1, dF1 = O.F_vt84f(np.array([1e-7]))
    assert F0[0] == 1.0
    assert abs(F1[0] - F0[0]) < 1e-6 and abs(dF1[0] - dF0[0]) < 1e-5
    assert abs(dF0[0] - float(-VT_MU + VT_ALPHA + mp.mpf(5) / 3)) < 1e-15
