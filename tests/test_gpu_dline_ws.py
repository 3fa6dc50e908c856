"""GPU parity of the derivative passes with warp-owned lines (the form
ofdft_autotune may pick; OFDFT_DLINE_WS starts a context with it): the GGA
energy and potential against the oracle for every tile shape the tuner
tries (1, 2 and 4 lines a warp), on a grid with radix-2, 3 and 5 axes and
a ragged last tile, in an orthorhombic and a sheared cell, and a
mixed-precision minimisation (its FP32 passes take the same form).

Bars as the other parity tests: energies 1e-10 of F_tot, the potential
1e-9 of its maximum; the mixed minimisation within the mixed form's
1e-6 Ha/atom.
"""
import numpy as np
import pytest

import oracle as O
from paper_1406_0835_gb300 import inputs, ofdft

pytestmark = pytest.mark.gpu

SHAPES = ["8,256", "8,128", "8,64", "16,256", "16,128"]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def random_phi(so, grid, seed):
    rng = np.random.default_rng(seed)
    return so.uniform_phi() * (1.0 + 0.1 * rng.standard_normal(grid))


def check_eval(ctx, so, phi):
    ev = O.evaluate(so, phi)
    E, v = ctx.energy_potential(phi)
    for k in ("F_tot", "F_s", "F_xc", "E_H"):
        assert abs(E[k] - ev[k]) <= 1e-10 * abs(ev["F_tot"]), (k, E[k], ev[k])
    assert np.max(np.abs(v - ev["v"])) <= 1e-9 * np.max(np.abs(ev["v"]))


@pytest.mark.parametrize("shape", SHAPES)
def test_warp_owned_lines_orthorhombic(shape, monkeypatch):
    monkeypatch.setenv("OFDFT_DLINE_WS", shape)
    cfg = inputs.config_single_point()
    grid = (30, 20, 24)     # pair columns: 20 * 12 = 240 and 30 * 12 = 360, ragged for 16-wide tiles
    so = O.System(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], "vt84f")
    with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], "vt84f") as ctx:
        check_eval(ctx, so, random_phi(so, grid, 7))


def test_warp_owned_lines_triclinic(monkeypatch):
    monkeypatch.setenv("OFDFT_DLINE_WS", "8,128")
    cfg = inputs.config_single_point()
    L = np.array(cfg["L"])
    cell = np.diag(L) + np.array([[0.0, 0.0, 0.0], [0.45, 0.0, 0.0], [-0.3, 0.55, 0.0]])
    ions = (cfg["ions"] / L) @ cell
    grid = (24, 20, 30)
    so = O.System(None, grid, ions, cfg["Z"], cfg["T"], "vt84f", cell=cell)
    with ofdft.Context(None, grid, ions, cfg["Z"], cfg["T"], "vt84f", cell=cell) as ctx:
        check_eval(ctx, so, random_phi(so, grid, 8))


def test_warp_owned_lines_mixed_minimisation(monkeypatch):
    monkeypatch.setenv("OFDFT_DLINE_WS", "16,128")
    d = inputs.hydrogen(16, 1.0, 3.125e4, 24, seed=2, functional="vt84f")
    grid = (24, 24, 24)
    so = O.System(d["L"], grid, d["ions"], d["Z"], d["T"], "vt84f")
    _, ev, _ = O.minimize(so, gtol=1e-10)
    with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], "vt84f", precision="mixed") as ctx:
        E, st = ctx.minimize(gtol=1e-8)
        assert st["status"] == 0 and st["evaluations_lo"] > 0
    assert abs(E["F_tot"] - ev["F_tot"]) / 16 < 1e-6


def test_warp_owned_lines_at_the_md_size(monkeypatch):
    """At the MD workload's size (96^3, 128 H, VT84F) the warp-synchronous
    derivative passes reproduce the block-synchronous ones: the same
    arithmetic in another order of threads, so energies agree to 1e-13 of
    F_tot and the potential to 1e-12 of its maximum."""
    d = inputs.config_md("vt84f")
    grid = d["grid"]
    rng = np.random.default_rng(12)
    phi = np.sqrt(128.0 / np.prod(d["L"])) * (1.0 + 0.05 * rng.standard_normal(grid))
    out = []
    for shape in (None, "16,128"):
        if shape:
            monkeypatch.setenv("OFDFT_DLINE_WS", shape)
        with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], "vt84f") as ctx:
            out.append(ctx.energy_potential(phi))
    (Ea, va), (Eb, vb) = out
    for k in ("F_tot", "F_s", "F_xc", "E_H"):
        assert abs(Ea[k] - Eb[k]) <= 1e-13 * abs(Ea["F_tot"]), k
    assert np.max(np.abs(va - vb)) <= 1e-12 * np.max(np.abs(va))
