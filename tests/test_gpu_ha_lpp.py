"""GPU parity with the Heine-Abarenkov hydrogen pseudopotential, Eq. (E4A).

Same bars as the Gaussian-ion parity tests: free energy 1e-10 relative,
potential 1e-9 of its range, density 1e-9, forces and pressure from the
converged density; the LPP pressure uses the stored dilation weights.
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


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("fn", ["fttf", "vt84f"])
@pytest.mark.parametrize("grid", [(16, 16, 16), (24, 20, 30)])
def test_energy_and_potential_match_oracle(fn, grid):
    cfg = inputs.config_single_point()
    rng = np.random.default_rng(7 + grid[1])
    so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn, lpp="ha")
    phi = so.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(grid))
    ev = O.evaluate(so, phi)
    with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn, lpp="ha") as ctx:
        E, v = ctx.energy_potential(phi)
    for k in ("F_tot", "F_s", "E_H", "E_loc", "F_xc", "E_ion"):
        assert abs(E[k] - ev[k]) <= 1e-10 * abs(ev["F_tot"]), (k, E[k], ev[k])
    for k in ("P", "P_loc"):
        assert abs(E[k] - ev[k]) <= 1e-9 * abs(ev["P"]), (k, E[k], ev[k])
    assert rel(E["E_alphaZ"], ev["E_alphaZ"]) < 1e-13
    assert np.max(np.abs(v - ev["v"])) <= 1e-9 * np.max(np.abs(ev["v"]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_minimisation_forces_pressure_match_oracle(precision):
    cfg = inputs.config_single_point()
    grid = (20, 20, 20)
    so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], "sga", lpp="ha")
    phi_o, ev_o, _ = O.minimize(so, gtol=1e-10)
    with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], "sga", lpp="ha",
                       precision=precision) as ctx:
        E, st = ctx.minimize(gtol=1e-10)
        assert st["status"] == 0
        assert rel(E["F_tot"], ev_o["F_tot"]) < 1e-10
        n = ctx.density()
        assert np.max(np.abs(n - ev_o["n"])) <= 1e-9 * np.max(ev_o["n"])
        F, P = ctx.forces()
    np.testing.assert_allclose(F, O.forces(so, ev_o), rtol=0, atol=1e-8)
    assert rel(P, ev_o["P"]) < 1e-8
