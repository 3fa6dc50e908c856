"""CPU: the pointwise functional the field kernels apply, evaluated on the
host through ofdft_pointwise_eval (same source as the kernels, no GPU).

Binary64 is pinned to the oracle's f_s (Eqs. (fTF), (FGGA), (vTF), (vftGGA))
and PZ81 (Sec. IV); the double-float form the FP64 kernels use by default
is pinned to binary64.  Errors are scaled to the size of the terms that
produce each output (f_s = tau0 xi F_tau - tau0 zeta F_sigma can cancel)."""
import numpy as np
import pytest

import oracle as O
from paper_1406_0835_gb300 import ofdft

OF_CS = 1.0 / (4.0 * (3.0 * np.pi ** 2) ** (2.0 / 3.0))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return ofdft.load()


def _points(seed, count=3000):
    # s^2 from 1e-9 (the enhancement factor's small-x series in the
    # double-float kernels) to 1e3 (its closed large-x form)
    rng = np.random.default_rng(seed)
    n = 10.0 ** rng.uniform(-5, 2, count)
    s2 = 10.0 ** rng.uniform(-9, 3, count)
    g2 = s2 * n ** (8.0 / 3.0) / OF_CS
    return n, g2


def _oracle(fn, n, g2, T_kelvin):
    T = T_kelvin * O.KB_HA_PER_K
    if fn == "fttf":
        d = O.fs_fttf(n, T)
        wc = np.zeros_like(n)
    else:
        gradn = np.stack([np.sqrt(g2), np.zeros_like(n), np.zeros_like(n)])
        d = O.fs_gga(n, gradn, T, O.FUNCTIONALS[fn])
        wc = d["W"][0] / gradn[0]
    eps, v = O.pz81(n)
    return dict(f=d["f"], ts=d["f_ent"], dfdn=d["dfdn"], wc=wc, eps=eps, vxc=v,
                scale=np.abs(d["f_kin"]) + np.abs(d["f_ent"]))


@pytest.mark.parametrize("fn", ["fttf", "sga", "vt84f", "kst2"])
@pytest.mark.parametrize("T_kelvin", [1.0e4, 3.125e4, 1.0e6])
def test_binary64_pointwise_matches_oracle(lib, fn, T_kelvin):
    n, g2 = _points(1)
    out, _ = ofdft.ofdft_pointwise_eval(fn, True, T_kelvin, n, g2, "f64")
    o = _oracle(fn, n, g2, T_kelvin)
    sc = o["scale"]
    # the temperature functions come from the piecewise fits (1e-13 in value,
    # 1e-10 in t-derivative); everything else is the same closed form
    assert np.max(np.abs(out[:, 0] - o["f"]) / sc) < 1e-12
    assert np.max(np.abs(out[:, 1] - o["ts"]) / sc) < 1e-12
    assert np.max(np.abs(out[:, 2] - o["dfdn"]) / (np.abs(o["dfdn"]) + sc / n)) < 1e-9
    if fn != "fttf":
        assert np.max(np.abs(out[:, 3] - o["wc"]) / np.abs(o["wc"])) < 1e-9
    assert np.max(np.abs(out[:, 4] - o["eps"]) / np.abs(o["eps"])) < 1e-13
    assert np.max(np.abs(out[:, 5] - o["vxc"]) / np.abs(o["vxc"])) < 1e-13


@pytest.mark.parametrize("fn", ["fttf", "sga", "vt84f", "kst2", "vwtf", "tw", "apbef"])
@pytest.mark.parametrize("T_kelvin", [2.0e3, 3.125e4, 4.0e6])
def test_double_float_pointwise_matches_binary64(lib, fn, T_kelvin):
    n, g2 = _points(2)
    a, used = ofdft.ofdft_pointwise_eval(fn, True, T_kelvin, n, g2, "f32x2")
    b, used64 = ofdft.ofdft_pointwise_eval(fn, True, T_kelvin, n, g2, "f64")
    assert used == n.size and used64 == 0
    sc = np.abs(b[:, 0]) + np.abs(b[:, 1])
    assert np.max(np.abs(a[:, 0] - b[:, 0]) / sc) < 1e-12
    assert np.max(np.abs(a[:, 1] - b[:, 1]) / sc) < 1e-12
    assert np.max(np.abs(a[:, 2] - b[:, 2]) / (np.abs(b[:, 2]) + sc / n)) < 1e-12
    if fn != "fttf":
        assert np.max(np.abs(a[:, 3] - b[:, 3]) / np.abs(b[:, 3])) < 5e-12
    assert np.max(np.abs(a[:, 4:] - b[:, 4:]) / np.abs(b[:, 4:])) < 1e-13


def test_double_float_domain_falls_back_to_binary64(lib):
    # n below 1e-18, s^2 above 1e10, t beyond the table (classical and
    # Sommerfeld ends): binary64 takes these points, bit for bit
    n = np.array([1e-20, 1e-3, 1e-12, 1e3])
    s2 = np.array([1.0, 1e12, 1.0, 1.0])
    g2 = s2 * n ** (8.0 / 3.0) / OF_CS
    for fn, T in (("vt84f", 4.0e6), ("fttf", 2.0e3)):
        a, used = ofdft.ofdft_pointwise_eval(fn, True, T, n, g2, "f32x2")
        b, _ = ofdft.ofdft_pointwise_eval(fn, True, T, n, g2, "f64")
        t = 2.0 * T * O.KB_HA_PER_K / (3.0 * np.pi ** 2 * n) ** (2.0 / 3.0)
        out = (n < 1e-18) | (t < 2.0 ** -20) | (t >= 2.0 ** 34)
        if fn != "fttf":
            out |= s2 > 1e10
        assert used == np.count_nonzero(~out)
        assert np.array_equal(a[out], b[out])
    with pytest.raises(ofdft.OfdftError):
        ofdft.ofdft_pointwise_eval("vt84f", True, 1e4, [1.0], [1.0], arith=7)


@pytest.mark.parametrize("fn", ["fttf", "vt84f"])
def test_double_float_over_the_whole_temperature_table(lib, fn):
    """Densities from 1e-16 to 1e6 bohr^-3 at 1e4 K and 1e6 K put the reduced
    temperature on every panel of the temperature table, [2^-20, 2^34) (the
    double-float Horner sums of xi and A take their high-degree terms in
    binary32), with the same bars against binary64."""
    rng = np.random.default_rng(9)
    for T in (1.0e4, 1.0e6):
        n = 10.0 ** rng.uniform(-16, 6, 20000)
        s2 = 10.0 ** rng.uniform(-9, 3, n.size)
        g2 = s2 * n ** (8.0 / 3.0) / OF_CS
        a, used = ofdft.ofdft_pointwise_eval(fn, True, T, n, g2, "f32x2")
        b, _ = ofdft.ofdft_pointwise_eval(fn, True, T, n, g2, "f64")
        assert used >= 0.9 * n.size
        sc = np.abs(b[:, 0]) + np.abs(b[:, 1])
        assert np.max(np.abs(a[:, 0] - b[:, 0]) / sc) < 1e-12
        assert np.max(np.abs(a[:, 1] - b[:, 1]) / sc) < 1e-12
        assert np.max(np.abs(a[:, 2] - b[:, 2]) / (np.abs(b[:, 2]) + sc / n)) < 1e-12
        if fn != "fttf":
            assert np.max(np.abs(a[:, 3] - b[:, 3]) / np.abs(b[:, 3])) < 5e-12
