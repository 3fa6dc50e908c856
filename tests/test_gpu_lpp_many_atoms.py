"""GPU parity of the structure-factor sums with many ions: v_ext(G) (through
E_loc and the potential) and the local-pseudopotential forces, Eq. (M12),
against the oracle, with more than one block of atoms (300 ions: two
chunks of 256) and grids whose even edges put points on every Nyquist
plane.  Orthorhombic with the Heine-Abarenkov ion of Eq. (E4A), and a
sheared (triclinic) cell with the Gaussian ion, where the partner of a
Nyquist point has its own form factor w(G').

Bars as the other parity tests: energies 1e-10 of F_tot, the potential
1e-9 of its maximum, forces 1e-8 Ha/bohr.
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


def normalised_phi(so, grid, seed):
    rng = np.random.default_rng(seed)
    phi = so.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(grid))
    dV = so.grid.omega / np.prod(grid)
    return phi * np.sqrt(np.sum(so.Z) / (np.sum(phi * phi) * dV))


def check(ctx, so, phi):
    ev = O.evaluate(so, phi)
    F_o = O.forces(so, ev)
    ctx.set_phi(phi)
    E, v = ctx.energy_potential()
    for k in ("F_tot", "E_loc", "E_H", "E_ion"):
        assert abs(E[k] - ev[k]) <= 1e-10 * abs(ev["F_tot"]), (k, E[k], ev[k])
    assert np.max(np.abs(v - ev["v"])) <= 1e-9 * np.max(np.abs(ev["v"]))
    F, _ = ctx.forces()
    assert np.max(np.abs(F - F_o)) <= 1e-8, np.max(np.abs(F - F_o))


def test_many_ions_orthorhombic_heine_abarenkov():
    grid = (40, 36, 32)
    d = inputs.hydrogen(300, 1.0, 3.125e4, 40, seed=21, functional="vt84f")
    so = O.System(d["L"], grid, d["ions"], d["Z"], d["T"], "vt84f", lpp="ha")
    phi = normalised_phi(so, grid, 4)
    with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], "vt84f", lpp="ha") as ctx:
        check(ctx, so, phi)


def test_many_ions_triclinic_gaussian():
    grid = (36, 40, 32)
    d = inputs.hydrogen(300, 1.0, 3.125e4, 40, seed=22, functional="sga")
    L = np.array(d["L"]) * np.ones(3)
    cell = np.diag(L) + np.array([[0.0, 0.0, 0.0], [0.45, 0.0, 0.0], [-0.3, 0.55, 0.0]])
    ions = (d["ions"] / L) @ cell
    so = O.System(None, grid, ions, d["Z"], d["T"], "sga", cell=cell)
    phi = normalised_phi(so, grid, 5)
    with ofdft.Context(None, grid, ions, d["Z"], d["T"], "sga", cell=cell) as ctx:
        check(ctx, so, phi)


def test_double_float_sums_match_binary64_sums_at_size():
    """At a size beyond the oracle's reach (512 ions, 96^3: two atom chunks,
    many row chunks), the double-float structure factor and forces match the
    binary64 kernels of a binary64 context on the same density: v_ext
    through E_loc within 1e-12 of F_tot, forces within 1e-9 Ha/bohr."""
    d = inputs.hydrogen(512, 2.0, 5.0e4, 96, seed=23, functional="sga")
    grid = (96, 96, 96)
    rng = np.random.default_rng(6)
    phi = np.sqrt(512.0 / np.prod(d["L"])) * (1.0 + 0.05 * rng.standard_normal(grid))
    res = []
    for pw in ("f32x2", "f64"):
        with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], "sga", pointwise=pw) as ctx:
            ctx.set_phi(phi)
            E, _ = ctx.energy_potential(want_v=False)
            F, _ = ctx.forces()
        res.append((E, F))
    (Ea, Fa), (Eb, Fb) = res
    assert abs(Ea["E_loc"] - Eb["E_loc"]) <= 1e-12 * abs(Eb["F_tot"])
    assert np.max(np.abs(Fa - Fb)) <= 1e-9
