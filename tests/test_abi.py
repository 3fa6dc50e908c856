"""C-ABI library checks that need no GPU: it builds, loads, exports every
entry point declared in include/ofdft.h, and its host-side temperature
tables agree with the oracle (kappa of footnote a of Table I, h~ of Eq. (s_s))."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1406_0835_gb300 import build as libbuild
from paper_1406_0835_gb300 import ofdft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return ofdft.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "ofdft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ofdft_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_entry_point(lib):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared calls
    assert sorted(ofdft.SIGNATURES) == names


def test_setup_rejects_bad_input_without_a_gpu(lib):
    # argument validation happens before any device call
    cfg_cell = np.diag([4.0, 4.0, 4.0])
    ions = np.zeros((1, 3))
    for grid, T, fn in (((14, 16, 16), 1e4, "fttf"),    # 14 = 2*7 is not {2,3,5}-smooth
                        ((15, 16, 16), 1e4, "fttf"),    # odd
                        ((16, 16, 16), -1.0, "fttf"),   # T <= 0
                        ((16, 16, 16), 1e4, 42)):       # unknown functional
        with pytest.raises(ofdft.OfdftError) as e:
            ofdft.ofdft_setup(cfg_cell, grid, ions, [1.0], T, fn)
        assert e.value.status == -1
    # general cells must be right-handed and finite (triclinic cells are accepted)
    left = np.array([[0.0, 4.0, 0.0], [4.0, 0.0, 0.0], [0.5, 0.0, 4.0]])
    bad = cfg_cell.copy()
    bad[1, 0] = np.nan
    for cell in (left, bad):
        with pytest.raises(ofdft.OfdftError) as e:
            ofdft.ofdft_setup(cell, (16, 16, 16), ions, [1.0], 1e4, "fttf")
        assert e.value.status == -1
    # FP64 arithmetic selector: only OFDFT_PW_F32X2 (0) and OFDFT_PW_F64 (1)
    p = ofdft.ofdft_default_params()
    assert p.pointwise == 0
    p.pointwise = 7
    with pytest.raises(ofdft.OfdftError) as e:
        ofdft.ofdft_setup(cfg_cell, (16, 16, 16), ions, [1.0], 1e4, "fttf", p)
    assert e.value.status == -1
    # local pseudopotential: Gaussian by default, Eq. (E4A)'s H values ready
    p = ofdft.ofdft_default_params()
    assert (p.lpp, p.lpp_A, p.lpp_qc) == (0, 6.18, 29.97)
    two = np.array([[0.0, 0.0, 0.0], [2.0, 2.0, 2.0]])
    for lpp, A, qc, Z in ((2, 6.18, 29.97, [1.0, 1.0]),             # unknown form
                          (1, 6.18, 0.0, [1.0, 1.0]),               # qc <= 0
                          (1, float("nan"), 29.97, [1.0, 1.0]),     # A not finite
                          (1, 6.18, 29.97, [1.0, 2.0])):            # two species
        p.lpp, p.lpp_A, p.lpp_qc = lpp, A, qc
        with pytest.raises(ofdft.OfdftError) as e:
            ofdft.ofdft_setup(cfg_cell, (16, 16, 16), two, Z, 1e4, "fttf", p)
        assert e.value.status == -1


def test_tabulated_temperature_functions_match_oracle(lib):
    rng = np.random.default_rng(0)
    t = np.concatenate([np.exp(rng.uniform(np.log(1e-6), np.log(1e10), 4000)),
                        np.logspace(-3, 2, 501), [2.0 ** -20, 2.0 ** 34 * 0.999]])
    out = ofdft.ofdft_tfunc_eval(t)
    z = O.xi_zeta(t)
    xi, zeta, h, dh, d2h = z["xi"], z["zeta"], z["h"], z["dh"], z["d2h"]
    A = (h - t * dh) / xi
    B = t * dh / zeta
    dA = -t * d2h / xi - (h - t * dh) * z["dxi"] / xi ** 2
    dB = (dh + t * d2h) / zeta - t * dh * z["dzeta"] / zeta ** 2
    # values: relative to what multiplies them in f_s = tau0 [xi F_tau - zeta F_sigma]
    assert np.max(np.abs(out[:, 0] - xi) / xi) < 1e-13
    assert np.max(np.abs(out[:, 1] - zeta) / xi) < 1e-13
    assert np.max(np.abs(out[:, 2] - A) / np.maximum(1.0, np.abs(A))) < 1e-13
    assert np.max(np.abs(out[:, 3] - B) * zeta / xi) < 1e-13
    # t-derivatives (polynomial derivatives of the fit), scaled the same way
    assert np.max(np.abs(out[:, 4] - z["dxi"]) * t / xi) < 1e-10
    assert np.max(np.abs(out[:, 5] - z["dzeta"]) * t / xi) < 1e-10
    assert np.max(np.abs(out[:, 6] - dA) * t / np.maximum(1.0, np.abs(A))) < 1e-10
    assert np.max(np.abs(out[:, 7] - dB) * t * zeta / xi) < 1e-10
    with pytest.raises(ofdft.OfdftError):
        ofdft.ofdft_tfunc_eval([0.0])


def test_missing_library_fails_loudly(tmp_path):
    saved = ofdft._lib
    try:
        ofdft._lib = None
        with pytest.raises(RuntimeError):
            ofdft.load(str(tmp_path / "nope.so"))
    finally:
        ofdft._lib = saved


def test_null_contexts_are_rejected_without_a_gpu(lib):
    """Entry points taking a context check it before any device call."""
    sig = np.zeros(9)
    assert lib.ofdft_stress(None, sig.ctypes.data_as(ofdft._P), None) == -1
    u, xi = np.zeros(2), np.zeros(6)
    n = ofdft.ctypes.c_int()
    assert lib.ofdft_md_andersen(None, 1e4, 0.5, u.ctypes.data_as(ofdft._P),
                                 xi.ctypes.data_as(ofdft._P), ofdft.ctypes.byref(n)) == -1
    assert lib.ofdft_forces(None, None, None) == -1
    assert b"NULL" in lib.ofdft_last_error(None)
