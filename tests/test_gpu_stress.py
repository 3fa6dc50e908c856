"""GPU parity of the stress tensor (Eq. (StressTensor)) through ofdft_stress.

Term by term against the oracle at the same density, to 1e-9 of the
largest entry of each term (the FP64 evaluation's bar for the pressure);
grids with Nyquist planes on every axis and a ragged y/x tile, both local
pseudopotentials.  At the minimised density -Tr Sigma/3 is the pressure
ofdft_forces reports.
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


@pytest.mark.parametrize("fn,lpp,grid", [
    ("vt84f", "gauss", (16, 16, 16)),
    ("sga", "ha", (24, 20, 30)),
    ("fttf", "gauss", (24, 20, 30)),
    ("fttf", "ha", (16, 16, 16)),
])
def test_stress_matches_oracle(fn, lpp, grid):
    cfg = inputs.config_single_point()
    so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn, lpp=lpp)
    rng = np.random.default_rng(21 + grid[2])
    phi = so.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(grid))
    phi *= np.sqrt(so.Ne / so.grid.integrate(phi * phi))
    ev = O.evaluate(so, phi)
    ref = O.stress(so, ev)
    with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn, lpp=lpp) as ctx:
        ctx.set_phi(phi)
        got = ctx.stress()
    for k in ("s", "xc", "H", "loc", "ion", "Sigma"):
        scale = np.max(np.abs(ref[k]))
        np.testing.assert_allclose(got[k], ref[k], rtol=0, atol=1e-9 * scale, err_msg=k)
    np.testing.assert_array_equal(got["Sigma"], got["Sigma"].T)


def test_stress_trace_is_the_pressure_at_equilibrium():
    cfg = inputs.config_single_point()
    with ofdft.Context(cfg["L"], (20, 20, 20), cfg["ions"], cfg["Z"], cfg["T"], "sga") as ctx:
        E, st = ctx.minimize(gtol=1e-9)
        F, P = ctx.forces()
        S = ctx.stress()["Sigma"]
    assert abs(-np.trace(S) / 3 - P) <= 1e-10 * abs(P)
    assert abs(-np.trace(S) / 3 - E["P"]) <= 1e-9 * abs(P)
