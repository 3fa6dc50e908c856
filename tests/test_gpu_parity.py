"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (FP64 path): free energy 1e-10 relative, density 1e-9 (max error
over max n), potential 1e-9 (max error over max |v|), forces 1e-9 hartree/bohr,
pressure 1e-9 relative; grid and ion index maps are exact (same seeded inputs,
same C-order layout).  The free-energy and density bars are the target the
method is built to; the others follow from the same arithmetic (double FFTs,
tabulated temperature functions accurate to ~1e-13).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1406_0835_gb300 import inputs, ofdft

pytestmark = pytest.mark.gpu

FUNCS = ["fttf", "sga", "vt84f", "kst2", "vwtf", "tw", "apbef"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def check_energy(E, ev, tol=1e-10):
    for k in ("F_tot", "F_s", "minus_TS", "E_H", "E_loc", "F_xc", "E_ion", "E_int"):
        assert abs(E[k] - ev[k]) <= tol * max(abs(ev["F_tot"]), 1.0), (k, E[k], ev[k])
    for k in ("P", "P_s", "P_xc", "P_H", "P_loc", "P_ion"):
        assert abs(E[k] - ev[k]) <= 1e-9 * max(abs(ev["P"]), 1e-6), (k, E[k], ev[k])


@pytest.mark.parametrize("fn", FUNCS)
@pytest.mark.parametrize("grid", [(16, 16, 16), (24, 20, 30), (40, 36, 32)])
def test_energy_and_potential_match_oracle(fn, grid):
    """One evaluation of Eqs. (E1)-(E4), (vTF)/(vftGGA), (vxc1) at a random density;
    the grids span several y/x tiles, ragged last tiles and odd pair counts per block."""
    cfg = inputs.config_single_point()
    rng = np.random.default_rng(abs(hash((fn, grid))) % 2 ** 32)
    so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn)
    phi = so.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(grid))
    ev = O.evaluate(so, phi)
    with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn) as ctx:
        E, v = ctx.energy_potential(phi)
        check_energy(E, ev)
        assert np.max(np.abs(v - ev["v"])) <= 1e-9 * np.max(np.abs(ev["v"]))
        # deterministic: a second evaluation is bit-identical
        E2, v2 = ctx.energy_potential(phi)
        assert E2["F_tot"] == E["F_tot"]
        assert np.array_equal(v, v2)


@pytest.mark.parametrize("fn", FUNCS)
def test_double_float_pointwise_matches_binary64(fn):
    """The FP64 kernels' default double-float pointwise functional against
    the binary64 one (ofdft_params.pointwise) on the same density: energies
    to 1e-12, potential to 1e-11 of its range; then both minimise to the
    same free energy."""
    cfg = inputs.config_mixed(2.5e5, grid=40, n_atoms=16)
    cfg["ions"] = cfg["ions"][:16]
    rng = np.random.default_rng(11)
    phi = np.sqrt(16.0 / np.prod(cfg["L"])) * (1.0 + 0.2 * rng.standard_normal(cfg["grid"]))
    out = {}
    for pw in ("f32x2", "f64"):
        with ofdft.Context(cfg["L"], cfg["grid"], cfg["ions"], cfg["Z"], cfg["T"], fn, pointwise=pw) as ctx:
            E, v = ctx.energy_potential(phi)
            Em, st = ctx.minimize(gtol=1e-8)
            assert st["status"] == 0
            out[pw] = (E, v, Em)
    (Ea, va, Ema), (Eb, vb, Emb) = out["f32x2"], out["f64"]
    for k in ("F_tot", "F_s", "minus_TS", "F_xc", "P", "P_s", "P_xc"):
        assert abs(Ea[k] - Eb[k]) <= 1e-12 * max(abs(Eb["F_tot"]), abs(Eb[k])), (k, Ea[k], Eb[k])
    assert np.max(np.abs(va - vb)) <= 1e-11 * np.max(np.abs(vb))
    assert rel(Ema["F_tot"], Emb["F_tot"]) <= 1e-11


@pytest.mark.parametrize("fn,tiny", [("fttf", 1e-11), ("vt84f", 1e-6)])
def test_double_float_kernels_fall_back_to_binary64(fn, tiny):
    """Points outside the double-float pointwise domain take the binary64
    routine inside the double-float kernels: n < 1e-18 (ftTF, phi = 1e-11 at
    every 97th point), s^2 > 1e10 (VT84F, phi = 1e-6 there) and t below the
    table at every point (0.1 K).  The result matches the binary64 kernels.
    (The VT84F potential then reaches 6e22; a density whose potential
    leaves the binary32 exponent range, 3.4e38, is outside what the
    double-float kernels represent.)"""
    cfg = inputs.config_single_point()
    grid = (16, 16, 16)
    rng = np.random.default_rng(5)
    for T in (cfg["T"], 0.1):
        so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], T, fn)
        phi = so.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(grid))
        phi.reshape(-1)[::97] = tiny
        out = {}
        for pw in ("f32x2", "f64"):
            with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], T, fn, pointwise=pw) as ctx:
                out[pw] = ctx.energy_potential(phi)
        (Ea, va), (Eb, vb) = out["f32x2"], out["f64"]
        assert abs(Ea["F_tot"] - Eb["F_tot"]) <= 1e-12 * abs(Eb["F_tot"]), (T, Ea["F_tot"], Eb["F_tot"])
        assert np.max(np.abs(va - vb)) <= 1e-11 * np.max(np.abs(vb)), T


def test_uniform_density_and_temperature_extremes():
    """s = 0 exactly (removable 0/0 of VT84F) and t over the table's range."""
    for T, rho in ((2.0e3, 10.0), (4.0e6, 0.1), (1.0e5, 1.0)):
        d = inputs.hydrogen(8, rho, T, 16, seed=7, functional="vt84f")
        so = O.System(d["L"], (16, 16, 16), d["ions"], d["Z"], T, "vt84f")
        with ofdft.Context(d["L"], (16, 16, 16), d["ions"], d["Z"], T, "vt84f") as ctx:
            E, v = ctx.energy_potential()
            ev = O.evaluate(so, so.uniform_phi())
            check_energy(E, ev)
            assert np.max(np.abs(v - ev["v"])) <= 1e-9 * np.max(np.abs(ev["v"]))


def test_single_point_minimisation_matches_oracle():
    """8 H, 1 g/cm^3, 100 kK, ftTF + PZ, 32^3: CG from the uniform start."""
    cfg = inputs.config_single_point()
    grid = cfg["grid"]
    so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], "fttf")
    phi_o, ev_o, st_o = O.minimize(so, gtol=1e-10)
    with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], "fttf") as ctx:
        E, st = ctx.minimize(gtol=1e-10)
        assert st["status"] == 0 and st["gnorm"] < 1e-10
        assert rel(E["F_tot"], ev_o["F_tot"]) < 1e-10
        n = ctx.density()
        assert np.max(np.abs(n - ev_o["n"])) <= 1e-9 * np.max(ev_o["n"])
        assert abs(np.sum(n) * so.grid.dV - so.Ne) < 1e-12 * so.Ne
        F, P = ctx.forces()
        np.testing.assert_allclose(F, O.forces(so, ev_o), rtol=0, atol=1e-9)
        assert rel(P, ev_o["P"]) < 1e-9
        assert abs(E["mu"] - st_o["mu"]) < 1e-9 * max(1.0, abs(st_o["mu"]))


@pytest.mark.parametrize("fn", ["sga", "vt84f"])
def test_gga_minimisation_matches_oracle(fn):
    cfg = inputs.config_single_point()
    grid = (20, 20, 20)
    so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn)
    phi_o, ev_o, _ = O.minimize(so, gtol=1e-10)
    with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn) as ctx:
        E, st = ctx.minimize(gtol=1e-10)
        assert st["status"] == 0
        assert rel(E["F_tot"], ev_o["F_tot"]) < 1e-10
        n = ctx.density()
        assert np.max(np.abs(n - ev_o["n"])) <= 1e-9 * np.max(ev_o["n"])
        F, P = ctx.forces()
        np.testing.assert_allclose(F, O.forces(so, ev_o), rtol=0, atol=1e-8)
        assert rel(P, ev_o["P"]) < 1e-8


def test_md_steps_match_oracle():
    """Velocity Verlet + Nose-Hoover with density extrapolation: first steps
    agree with the oracle's integrator (chaos makes later steps diverge)."""
    d = inputs.hydrogen(8, 1.0, 3.125e4, 16, seed=2, functional="sga", vel_seed=3)
    grid = (16, 16, 16)
    so = O.System(d["L"], grid, d["ions"], d["Z"], d["T"], "sga")
    st = O.MDState(d["ions"], d["vel"], d["masses"], d["T"], dt_fs=0.2)
    O.md_prepare(so, st, gtol=1e-10)
    with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], "sga") as ctx:
        out = ctx.md_step(0.2, d["T"], nsteps=0, pos=d["ions"] + 1e-3, vel=d["vel"], gtol=1e-10)
        out = ctx.md_step(0.2, d["T"], nsteps=0, pos=d["ions"], vel=d["vel"], gtol=1e-10)
        np.testing.assert_allclose(out["F"], st.F, atol=1e-8)
        for step in range(3):
            O.md_step(so, st, gtol=1e-10)
            out = ctx.md_step(0.2, d["T"], nsteps=1, gtol=1e-10)
        pos, vel = ctx.md_state()
        np.testing.assert_allclose(pos, st.R, rtol=0, atol=1e-10)
        np.testing.assert_allclose(vel, st.V, rtol=0, atol=1e-12)
        np.testing.assert_allclose(out["F"], st.F, rtol=0, atol=1e-8)
        assert rel(out["E"]["F_tot"], st.ev["F_tot"]) < 1e-10
        assert rel(ctx.md_conserved(), O.md_conserved(st)) < 1e-10
        # passing back the returned state continues the same trajectory
        out2 = ctx.md_step(0.2, d["T"], nsteps=1, pos=pos, vel=vel, gtol=1e-10)
        O.md_step(so, st, gtol=1e-10)
        np.testing.assert_allclose(out2["pos"], st.R, rtol=0, atol=1e-10)


@pytest.mark.parametrize("fn", ["fttf", "vt84f"])
@pytest.mark.parametrize("grid,L,nat", [
    ((512, 8, 8), (40.0, 3.0, 3.0), 3),      # longest supported axis (8 x 8 x 8 stages)
    ((10, 12, 18), (3.0, 3.5, 4.5), 1),      # radix-5 and radix-3 axes, orthorhombic cell, one ion
    ((8, 8, 8), (2.2, 2.2, 2.2), 2),         # smallest grid
])
def test_edge_shapes_match_oracle(fn, grid, L, nat):
    """Edge shapes: the maximum axis length, radices 3 and 5 on an
    orthorhombic cell, the minimum grid, one and two ions."""
    rng = np.random.default_rng(sum(grid) + nat)
    ions = rng.uniform(0, 1, (nat, 3)) * np.asarray(L)
    Z = np.ones(nat)
    so = O.System(L, grid, ions, Z, 5.0e4, fn)
    phi = so.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(grid))
    ev = O.evaluate(so, phi)
    with ofdft.Context(L, grid, ions, Z, 5.0e4, fn) as ctx:
        E, v = ctx.energy_potential(phi)
        check_energy(E, ev)
        assert np.max(np.abs(v - ev["v"])) <= 1e-9 * np.max(np.abs(ev["v"]))


def test_invalid_inputs_are_rejected():
    cfg = inputs.config_single_point()
    with pytest.raises(ofdft.OfdftError):
        ofdft.Context(cfg["L"], (18, 18, 14), cfg["ions"], cfg["Z"], cfg["T"], "fttf")
    with ofdft.Context(cfg["L"], (8, 8, 8), cfg["ions"], cfg["Z"], cfg["T"], "fttf") as ctx:
        with pytest.raises(ofdft.OfdftError):
            ctx.minimize(gtol=-1.0)
        bad = np.full(512, np.nan)
        with pytest.raises(ofdft.OfdftError):
            ctx.energy_potential(bad)
        E, st = ctx.minimize(gtol=1e-8)        # 8^3: the smallest grid still works
        assert st["status"] == 0


def test_full_size_md_workload_sampled():
    """128 H, 96^3, VT84F + PZ, FP64 (the MD workload): one evaluation compared
    element by element with the oracle, then a GPU minimisation whose result
    the oracle confirms is a stationary point (Euler equation, Eq. (E10))."""
    d = inputs.config_md("vt84f")
    grid = d["grid"]
    so = O.System(d["L"], grid, d["ions"], d["Z"], d["T"], "vt84f")
    rng = np.random.default_rng(21)
    phi = so.uniform_phi() * (1.0 + 0.05 * rng.standard_normal(grid))
    ev = O.evaluate(so, phi)
    with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], "vt84f") as ctx:
        E, v = ctx.energy_potential(phi)
        check_energy(E, ev)
        assert np.max(np.abs(v - ev["v"])) <= 1e-9 * np.max(np.abs(ev["v"]))
        E, st = ctx.minimize(gtol=1e-8)
        assert st["status"] == 0
        n = ctx.density()
        ev2 = O.evaluate(so, np.sqrt(n))
        assert rel(E["F_tot"], ev2["F_tot"]) < 1e-10
        phi2 = np.sqrt(n)
        mu = float(np.sum(phi2 * phi2 * ev2["v"]) / np.sum(phi2 * phi2))
        g = 2.0 * phi2 * (ev2["v"] - mu)
        assert math.sqrt(so.grid.dV * float(np.sum(g * g))) < 2e-8
        F, P = ctx.forces()
        np.testing.assert_allclose(F, O.forces(so, ev2), rtol=0, atol=1e-8)
        assert rel(P, ev2["P"]) < 1e-9
