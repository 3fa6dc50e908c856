"""GPU truncated Newton (ofdft_minimize_tn), the alternative to CG that
Sec. II names, against the oracle's minimize_tn and CG minimum.

Both minimisers reach the minimiser of the same discrete functional, so
the bars are the FP64 parity bars of the CG tests: free energy 1e-10
relative, density 1e-9 of its maximum, forces 1e-8 Ha/bohr, pressure 1e-8
relative."""
import numpy as np
import pytest

import oracle as O
from paper_1406_0835_gb300 import inputs, ofdft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("fn,precision", [("sga", "fp64"), ("vt84f", "fp64"), ("vt84f", "mixed"), ("fttf", "fp64")])
def test_truncated_newton_matches_oracle(fn, precision):
    cfg = inputs.config_single_point()
    grid = (20, 20, 20)
    so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn)
    _, ev_tn, st_tn = O.minimize_tn(so, gtol=1e-10)
    _, ev_cg, _ = O.minimize(so, gtol=1e-10)
    assert st_tn["status"] == "converged"
    assert rel(ev_tn["F_tot"], ev_cg["F_tot"]) < 1e-11        # the oracle's two minimisers agree
    with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn, precision=precision) as ctx:
        E, st, nh = ctx.minimize_tn(gtol=1e-10)
        assert st["status"] == 0 and st["gnorm"] < 1e-10 and nh > 0
        assert st["evaluations"] >= 1 + 2 * nh
        assert rel(E["F_tot"], ev_tn["F_tot"]) < 1e-10
        n = ctx.density()
        assert np.max(np.abs(n - ev_tn["n"])) <= 1e-9 * np.max(ev_tn["n"])
        assert abs(np.sum(n) * so.grid.dV - so.Ne) < 1e-12 * so.Ne
        F, P = ctx.forces()
    np.testing.assert_allclose(F, O.forces(so, ev_tn), rtol=0, atol=1e-8)
    assert rel(P, ev_tn["P"]) < 1e-8
    # the same algorithm on both sides: the outer iteration counts agree closely
    assert abs(st["iterations"] - st_tn["iterations"]) <= max(2, st_tn["iterations"] // 5)


def test_truncated_newton_arguments():
    cfg = inputs.config_single_point(grid=16)
    with ofdft.Context(cfg["L"], (16, 16, 16), cfg["ions"], cfg["Z"], cfg["T"], "sga") as ctx:
        for kw in (dict(gtol=-1.0), dict(maxit=0), dict(inner_max=0), dict(eta=1.5), dict(eta=0.0)):
            with pytest.raises(ofdft.OfdftError) as e:
                ctx.minimize_tn(**kw)
            assert e.value.status == -1
        E, st, nh = ctx.minimize_tn(gtol=1e-6, maxit=1, raise_on_noconv=False)
        assert st["status"] == -3 and st["iterations"] == 1
