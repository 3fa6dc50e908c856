"""Pins for the oracle's stress tensor (Eqs. (StressTensor), (pressure),
(stressTF_a), (stressTF_b), (stressLSDAxc)) and for the general-cell grid
and Ewald sum it is checked with.

The stress tensor is pinned by finite differences of the minimised free
energy under homogeneous strains, shears included (a sheared cell is
triclinic, hence the general-cell grid); that grid is pinned to the
orthorhombic one, to the exact-derivative property, and the general Ewald
sum to the textbook bcc Madelung energy in the primitive (triclinic) cell.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1406_0835_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SHEARED = np.array([[4.4, 0.0, 0.0], [0.7, 4.2, 0.0], [-0.5, 0.4, 4.6]])


def test_cell_grid_reduces_to_orthorhombic():
    L = (4.0, 5.0, 6.0)
    a, b = O.Grid(L, (12, 10, 8)), O.CellGrid(np.diag(L), (12, 10, 8))
    for x, y in ((a.G2, b.G2), (a.Gx, b.Gx), (a.Gy, b.Gy), (a.Gz, b.Gz),
                 (a.Dx, b.Dx), (a.Dy, b.Dy), (a.Dz, b.Dz)):
        np.testing.assert_allclose(np.broadcast_to(x, a.shape), y, rtol=1e-14, atol=1e-14)
    assert b.omega == pytest.approx(a.omega, rel=1e-15)


def test_cell_grid_gradient_divergence_adjoint_and_plane_waves():
    g = O.CellGrid(SHEARED, (12, 10, 14))
    rng = np.random.default_rng(4)
    n = rng.standard_normal(g.shape)
    W = rng.standard_normal((3,) + g.shape)
    assert np.sum(g.grad(n) * W) == pytest.approx(-np.sum(n * g.div(W)), rel=1e-12)
    # the gradient of a resolved plane wave cos(G.r) is -G sin(G.r)
    frac = np.stack(np.meshgrid(*[np.arange(m) / m for m in g.shape], indexing="ij"), -1)
    r = frac @ g.cell
    k = np.array([1, -2, 3])
    G = k @ g.B
    f = np.cos(r @ G)
    gr = g.grad(f)
    for a in range(3):
        np.testing.assert_allclose(gr[a], -G[a] * np.sin(r @ G), atol=1e-11)


def test_ewald_cell_matches_orthorhombic_and_bcc_madelung():
    L = [3.0, 4.0, 5.0]
    R = np.array([[0.1, 0.2, 0.3], [1.5, 2.1, 3.3], [2.9, 0.1, 4.0]])
    Z = [1.0, 2.0, 1.0]
    E0, F0 = O.ewald(L, R, Z)
    E1, F1, _ = O.ewald_cell(np.diag(L), R, Z)
    assert E1 == pytest.approx(E0, rel=1e-12)
    np.testing.assert_allclose(F1, F0, atol=1e-11)
    gold = json.load(open(os.path.join(GOLD, "madelung.json")))
    a = 2.0
    prim = 0.5 * a * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]])
    E, F, _ = O.ewald_cell(prim, [[0.3, 0.1, 0.2]], [1.0])
    rws = (3.0 * a ** 3 / 2.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
    assert E * rws == pytest.approx(gold["bcc_energy_per_ion_times_rws"], rel=1e-11)
    # the same lattice in another basis (a_2 -> a_2 + a_1) has the same energy
    prim2 = prim.copy()
    prim2[1] += prim[0]
    assert O.ewald_cell(prim2, [[0.3, 0.1, 0.2]], [1.0])[0] == pytest.approx(E, rel=1e-12)


def _strained(cell, R, eps):
    M = np.eye(3) + eps
    return cell @ M.T, np.asarray(R) @ M.T


def _eps(a, b, d):
    e = np.zeros((3, 3))
    e[a, b] += 0.5 * d
    e[b, a] += 0.5 * d
    return e


@pytest.mark.parametrize("ab", [(0, 0), (0, 1), (1, 2), (2, 0)])
def test_ewald_stress_is_strain_derivative(ab):
    R = np.array([[0.1, 0.2, 0.3], [1.5, 2.1, 3.3], [2.9, 0.1, 4.0], [3.7, 2.2, 1.0]])
    Z = [1.0, 2.0, 1.0, 3.0]
    E, F, S = O.ewald_cell(SHEARED, R, Z)
    V = abs(np.linalg.det(SHEARED))
    d = 1e-5
    Ep = O.ewald_cell(*_strained(SHEARED, R, _eps(*ab, d)), Z, alpha=1.1)[0]
    Em = O.ewald_cell(*_strained(SHEARED, R, _eps(*ab, -d)), Z, alpha=1.1)[0]
    assert (Ep - Em) / (2 * d) / V == pytest.approx(S[ab], rel=1e-7, abs=1e-10)
    np.testing.assert_allclose(S, S.T, atol=1e-14)
    assert -np.trace(S) / 3 == pytest.approx(E / (3 * V), rel=1e-11)   # Coulomb homogeneity


def test_cell_grid_potential_is_derivative_of_discrete_energy():
    cfg = I.config_single_point()
    cell = np.diag(cfg["L"]) + np.array([[0.0, 0.0, 0.0], [0.6, 0.0, 0.0], [-0.3, 0.5, 0.0]])
    s = O.System(None, (12, 12, 12), cfg["ions"], cfg["Z"], 1e5, "sga", cell=cell)
    rng = np.random.default_rng(3)
    phi = s.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(s.grid.shape))
    ev = O.evaluate(s, phi)
    n = phi * phi
    for j in [(0, 0, 0), (3, 5, 7), (11, 2, 9)]:
        h = 1e-4 * n[j]
        F = []
        for k in (-2, -1, 1, 2):
            nn = n.copy()
            nn[j] += k * h
            F.append(O.evaluate(s, np.sqrt(nn))["F_tot"])
        d = (F[0] - 8 * F[1] + 8 * F[2] - F[3]) / (12 * h) / s.grid.dV
        assert d == pytest.approx(ev["v"][j], rel=2e-8, abs=1e-9)


def _F_min(cell, R, fn, lpp, phi0):
    cfg = I.config_single_point()
    s = O.System(None, (12, 12, 12), R, cfg["Z"], 1e5, fn, lpp=lpp, cell=cell)
    phi, ev, _ = O.minimize(s, phi0, gtol=1e-11)
    return s, phi, ev


@pytest.mark.parametrize("fn,lpp,comps", [
    ("sga", "gauss", [(0, 0), (0, 1), (1, 2)]),
    ("fttf", "ha", [(2, 2), (0, 2)]),
])
def test_stress_is_strain_derivative_of_minimised_energy(fn, lpp, comps):
    """Eq. (StressTensor): V Sigma_ab = dF/d eps_ab at electronic equilibrium,
    fractional coordinates fixed; shears make the cell triclinic."""
    cfg = I.config_single_point()
    cell0 = np.diag(cfg["L"])
    s, phi, ev = _F_min(cell0, cfg["ions"], fn, lpp, None)
    S = O.stress(s, ev)
    np.testing.assert_allclose(S["Sigma"], S["Sigma"].T, atol=1e-13)
    assert -np.trace(S["Sigma"]) / 3 == pytest.approx(ev["P"], rel=1e-12)
    V = s.grid.omega
    d = 1e-4
    for ab in comps:
        Fp = _F_min(*_strained(cell0, cfg["ions"], _eps(*ab, d)), fn, lpp, phi)[2]["F_tot"]
        Fm = _F_min(*_strained(cell0, cfg["ions"], _eps(*ab, -d)), fn, lpp, phi)[2]["F_tot"]
        fd = (Fp - Fm) / (2 * d) / V
        assert fd == pytest.approx(S["Sigma"][ab], rel=2e-6, abs=2e-8), ab


def test_stress_in_a_triclinic_cell():
    """The same strain derivative starting from a sheared cell (GGA, Gaussian ion)."""
    cfg = I.config_single_point()
    cell0 = np.diag(cfg["L"]) + np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, -0.4, 0.0]])
    frac = cfg["ions"] / np.array(cfg["L"])
    R0 = frac @ cell0
    s, phi, ev = _F_min(cell0, R0, "vt84f", "gauss", None)
    S = O.stress(s, ev)
    V = s.grid.omega
    d = 1e-4
    for ab in ((0, 1), (1, 1)):
        Fp = _F_min(*_strained(cell0, R0, _eps(*ab, d)), "vt84f", "gauss", phi)[2]["F_tot"]
        Fm = _F_min(*_strained(cell0, R0, _eps(*ab, -d)), "vt84f", "gauss", phi)[2]["F_tot"]
        assert (Fp - Fm) / (2 * d) / V == pytest.approx(S["Sigma"][ab], rel=2e-6, abs=2e-8), ab


def test_stress_rotates_as_a_tensor():
    """A rigid rotation of cell and ions leaves the discrete free energy
    unchanged (the grid lives in fractional coordinates) and rotates the
    stress tensor: Sigma' = Q Sigma Q^T."""
    cfg = I.config_single_point()
    cell0 = np.diag(cfg["L"]) + np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, -0.4, 0.0]])
    R0 = (cfg["ions"] / np.array(cfg["L"])) @ cell0
    th = 0.37
    Q = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    Q = Q @ np.array([[1.0, 0.0, 0.0], [0.0, np.cos(0.8), -np.sin(0.8)], [0.0, np.sin(0.8), np.cos(0.8)]])
    out = []
    for cell, R in ((cell0, R0), (cell0 @ Q.T, R0 @ Q.T)):
        s = O.System(None, (12, 12, 12), R, cfg["Z"], 1e5, "vt84f", cell=cell)
        rng = np.random.default_rng(8)
        phi = s.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(s.grid.shape))
        ev = O.evaluate(s, phi)
        out.append((ev, O.stress(s, ev), O.forces(s, ev)))
    (e0, s0, f0), (e1, s1, f1) = out
    assert e1["F_tot"] == pytest.approx(e0["F_tot"], rel=1e-12)
    np.testing.assert_allclose(s1["Sigma"], Q @ s0["Sigma"] @ Q.T, atol=1e-12 * np.max(np.abs(s0["Sigma"])))
    np.testing.assert_allclose(f1, f0 @ Q.T, atol=1e-11 * np.max(np.abs(f0)))
