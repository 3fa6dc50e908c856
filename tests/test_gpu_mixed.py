"""Mixed precision (FP32 FFTs and pointwise terms, FP64 reductions, line
search, Ewald, forces and a final FP64 evaluation) against the FP64 path.

Workload: 256 H at 4.0 g/cm^3, VT84F + PZ, 128^3, T in {10 kK, 250 kK, 4 MK}.
Tolerances stated for this form: free energy within 1e-6 Ha/atom, forces
within 1e-4 Ha/bohr, pressure within 1e-3 relative, both against the FP64 GPU
minimisation (itself parity-tested against the oracle) and, for the energy
and pressure, against the oracle evaluated at the mixed-precision density.
"""
import numpy as np
import pytest

import oracle as O
from paper_1406_0835_gb300 import inputs, ofdft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("T", [1.0e4, 2.5e5, 4.0e6])
@pytest.mark.parametrize("gtol", [1e-8, ofdft.MIXED_FORM_GTOL])
def test_mixed_precision_against_fp64(T, gtol):
    """The mixed form at the plain tolerance and at the looser one the batched
    and serving forms use: both meet the stated per-result tolerances."""
    d = inputs.config_mixed(T)
    nat = len(d["Z"])
    res = {}
    for prec in ("fp64", "mixed"):
        with ofdft.Context(d["L"], d["grid"], d["ions"], d["Z"], T, "vt84f", precision=prec) as ctx:
            E, st = ctx.minimize(gtol=1e-8 if prec == "fp64" else gtol, maxit=20000, raise_on_noconv=False)
            assert st["status"] == 0, st
            if prec == "mixed":
                assert st["evaluations_lo"] > 0
            F, P = ctx.forces()
            res[prec] = (E, F, P, ctx.density())
    E64, F64, P64, n64 = res["fp64"]
    E32, F32, P32, n32 = res["mixed"]
    assert abs(E32["F_tot"] - E64["F_tot"]) / nat < 1e-6
    assert np.max(np.abs(F32 - F64)) < 1e-4
    assert abs(P32 - P64) <= 1e-3 * abs(P64)
    # the oracle's FP64 evaluation at the mixed-precision density
    so = O.System(d["L"], d["grid"], d["ions"], d["Z"], T, "vt84f")
    ev = O.evaluate(so, np.sqrt(n32).reshape(d["grid"]))
    assert abs(E32["F_tot"] - ev["F_tot"]) <= 1e-10 * abs(ev["F_tot"])
    assert abs(P32 - ev["P"]) <= 1e-9 * abs(ev["P"])
