"""GPU parity in a general (triclinic) cell against the oracle's general-cell
grid and Ewald sum: energy and potential at a random density, then the
minimised density, forces and stress tensor.  Same bars as the
orthorhombic parity tests.
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


def sheared():
    cfg = inputs.config_single_point()
    L = np.array(cfg["L"])
    cell = np.diag(L) + np.array([[0.0, 0.0, 0.0], [0.45, 0.0, 0.0], [-0.3, 0.55, 0.0]])
    ions = (cfg["ions"] / L) @ cell
    return cfg, cell, ions


@pytest.mark.parametrize("fn,grid", [("fttf", (16, 16, 16)), ("vt84f", (24, 20, 30))])
def test_energy_and_potential_match_oracle(fn, grid):
    cfg, cell, ions = sheared()
    so = O.System(None, grid, ions, cfg["Z"], cfg["T"], fn, cell=cell)
    rng = np.random.default_rng(5 + grid[2])
    phi = so.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(grid))
    ev = O.evaluate(so, phi)
    with ofdft.Context(None, grid, ions, cfg["Z"], cfg["T"], fn, cell=cell) as ctx:
        E, v = ctx.energy_potential(phi)
    for k in ("F_tot", "F_s", "E_H", "E_loc", "F_xc", "E_ion"):
        assert abs(E[k] - ev[k]) <= 1e-10 * abs(ev["F_tot"]), (k, E[k], ev[k])
    assert abs(E["P"] - ev["P"]) <= 1e-9 * abs(ev["P"])
    assert np.max(np.abs(v - ev["v"])) <= 1e-9 * np.max(np.abs(ev["v"]))


def test_minimisation_forces_stress_match_oracle():
    cfg, cell, ions = sheared()
    grid = (20, 20, 20)
    so = O.System(None, grid, ions, cfg["Z"], cfg["T"], "sga", cell=cell)
    phi_o, ev_o, _ = O.minimize(so, gtol=1e-10)
    S_o = O.stress(so, ev_o)
    with ofdft.Context(None, grid, ions, cfg["Z"], cfg["T"], "sga", cell=cell) as ctx:
        E, st = ctx.minimize(gtol=1e-10)
        assert st["status"] == 0
        assert rel(E["F_tot"], ev_o["F_tot"]) < 1e-10
        n = ctx.density()
        assert np.max(np.abs(n - ev_o["n"])) <= 1e-9 * np.max(ev_o["n"])
        F, P = ctx.forces()
        S = ctx.stress()
    np.testing.assert_allclose(F, O.forces(so, ev_o), rtol=0, atol=1e-8)
    assert rel(P, ev_o["P"]) < 1e-8
    for k in ("s", "xc", "H", "loc", "ion", "Sigma"):
        np.testing.assert_allclose(S[k], S_o[k], rtol=0, atol=1e-8 * np.max(np.abs(S_o[k])), err_msg=k)
