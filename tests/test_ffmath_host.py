"""CPU: the double-float primitives of the FP64 field kernels (sum, product,
quotient, square root, exp, e^x - 1, ln, x^(-1/3)), compiled for the host
from the kernels' source and checked against 40-digit references on the
exact double-float inputs.  Bounds in units of u^2 = 2^-48 (u = 2^-24, the
binary32 unit roundoff): the error-free-transformation algorithms named in
ffmath.cuh guarantee a few u^2 while every part stays a normal binary32;
near the ends of the binary32 exponent range the low word loses bits.
The host's binary32 seeds (division, sqrtf, logf, 1/cbrtf) may differ from
the device's by an ulp; the correction steps absorb that."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from paper_1406_0835_gb300 import ofdft  # noqa: E402

U2 = 2.0 ** -48


@pytest.fixture(scope="module", autouse=True)
def lib():
    import __graft_entry__
    __graft_entry__.build()
    mp.mp.dps = 40
    return ofdft.load()


def dd(x):
    """Nearest double-float of each binary64 (hi = float(x), lo = float(x - hi))."""
    hi = np.float32(x).astype(np.float64)
    return hi + np.float32(x - hi).astype(np.float64)


def max_rel(got, ref, floor=None):
    worst = 0.0
    for g, r in zip(got, ref):
        den = abs(r) if floor is None else max(abs(r), floor)
        worst = max(worst, float(abs(mp.mpf(float(g)) - r) / den))
    return worst


def operands(seed, n=3000, decades=12):
    rng = np.random.default_rng(seed)
    x = dd(rng.uniform(-1, 1, n) * 10.0 ** rng.uniform(-decades, decades, n))
    y = dd(rng.uniform(-1, 1, n) * 10.0 ** rng.uniform(-decades, decades, n))
    return rng, x, y


def test_sum_product_quotient():
    rng, x, y = operands(1)
    yc = y.copy()
    yc[:800] = dd(-x[:800] * (1.0 + rng.uniform(-1e-6, 1e-6, 800)))   # cancellation
    m = [mp.mpf(float(a)) for a in x]
    assert max_rel(ofdft.ofdft_ffmath_eval("add", x, yc), [a + mp.mpf(float(b)) for a, b in zip(m, yc)]) < 3 * U2
    assert max_rel(ofdft.ofdft_ffmath_eval("mul", x, y), [a * mp.mpf(float(b)) for a, b in zip(m, y)]) < 5 * U2
    assert max_rel(ofdft.ofdft_ffmath_eval("div", x, y), [a / mp.mpf(float(b)) for a, b in zip(m, y)]) < 8 * U2


def test_sqrt_and_inverse_cube_root():
    rng = np.random.default_rng(2)
    x = dd(10.0 ** rng.uniform(-18, 18, 3000))
    m = [mp.mpf(float(a)) for a in x]
    assert max_rel(ofdft.ofdft_ffmath_eval("sqrt", x), [mp.sqrt(a) for a in m]) < 4 * U2
    assert max_rel(ofdft.ofdft_ffmath_eval("rcbrt", x), [a ** (-mp.mpf(1) / 3) for a in m]) < 6 * U2


def test_exp_expm1_log():
    rng = np.random.default_rng(3)
    x = dd(rng.uniform(-60.0, 60.0, 3000))
    assert max_rel(ofdft.ofdft_ffmath_eval("exp", x), [mp.exp(mp.mpf(float(a))) for a in x]) < 4 * U2
    # e^x - 1 for x <= 0, from the reduced series near 0 to e^x - 1 far out
    xm = dd(-10.0 ** rng.uniform(-12, 1.9, 3000))
    assert max_rel(ofdft.ofdft_ffmath_eval("expm1_neg", xm), [mp.expm1(mp.mpf(float(a))) for a in xm]) < 6 * U2
    # ln x: a few u^2 of max(1, |ln x|), including x near 1 where ln x -> 0
    xl = np.concatenate([dd(10.0 ** rng.uniform(-25, 25, 2000)), dd(1.0 + rng.uniform(-1e-3, 1e-3, 1000))])
    ref = [mp.log(mp.mpf(float(a))) for a in xl]
    got = ofdft.ofdft_ffmath_eval("log", xl)
    worst = max(float(abs(mp.mpf(float(g)) - r) / max(1, abs(r))) for g, r in zip(got, ref))
    assert worst < 3 * U2
    # below e^-87 the routine returns 0 (documented; the functional's terms there are negligible)
    assert ofdft.ofdft_ffmath_eval("exp", np.array([-90.0]))[0] == 0.0
    with pytest.raises(ofdft.OfdftError):
        ofdft.ofdft_ffmath_eval(9, np.array([1.0]))


def test_binary_operations_check_the_second_operand():
    """add, mul and div read y[i] for every x[i]: a missing or shorter y is
    refused before the library is called."""
    x = np.linspace(1.0, 2.0, 8)
    for op in ("add", "mul", "div"):
        with pytest.raises(ValueError):
            ofdft.ofdft_ffmath_eval(op, x, x[:3])
        with pytest.raises(ValueError):
            ofdft.ofdft_ffmath_eval(op, x)
    assert ofdft.ofdft_ffmath_eval("sqrt", x).shape == x.shape
