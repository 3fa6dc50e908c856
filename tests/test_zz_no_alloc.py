"""The allocation-free entry point, ofdft_energy_potential_static.

It serves callers that must not allocate device memory (latency-critical
loops where cudaMalloc may synchronise the GPU, programs whose device memory
belongs to another allocator).  Its results must equal those of the regular
entry point, ofdft_setup + ofdft_energy_potential, within the tolerances of
the parity tests: free energy 1e-10 relative, potential 1e-9 of max |v|.
Two calls in a row check that the shared scratch array is reused correctly.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1406_0835_gb300 import inputs, ofdft

pytestmark = pytest.mark.gpu


def test_static_entry_point_matches_context_path():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    cfg = inputs.config_single_point()
    rng = np.random.default_rng(123)
    cases = [("fttf", (32, 32, 32)), ("vt84f", (24, 20, 30))]    # two calls in a row
    for fn, grid in cases:
        N = int(np.prod(grid))
        phi = np.sqrt(8.0 / np.prod(cfg["L"])) * (1.0 + 0.1 * rng.standard_normal(N))
        with ofdft.Context(cfg["L"], grid, cfg["ions"], cfg["Z"], cfg["T"], fn) as ctx:
            E_ref, v_ref = ctx.energy_potential(phi)
        phi_d = torch.tensor(phi, dtype=torch.float64, device="cuda")
        v_d = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        E = ofdft.ofdft_energy_potential_static(np.diag(cfg["L"]), grid, cfg["ions"], cfg["Z"],
                                                cfg["T"], fn, phi_d.data_ptr(), v_d.data_ptr())
        v = v_d.cpu().numpy().reshape(grid)
        for k in ("F_tot", "F_s", "minus_TS", "E_H", "E_loc", "F_xc", "E_ion", "P"):
            assert abs(E[k] - E_ref[k]) <= 1e-10 * max(abs(E_ref["F_tot"]), 1.0), (fn, k, E[k], E_ref[k])
        assert np.max(np.abs(v - v_ref)) <= 1e-9 * np.max(np.abs(v_ref)), fn
    # sizes beyond the fixed scratch are rejected with a clear error
    big = torch.zeros(64 * 64 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(ofdft.OfdftError) as e:
        ofdft.ofdft_energy_potential_static(np.diag(cfg["L"]), (64, 64, 64), cfg["ions"], cfg["Z"],
                                            cfg["T"], "fttf", big.data_ptr(), big.data_ptr())
    assert e.value.status == -1


def test_static_entry_point_at_its_limits():
    """The largest systems the fixed scratch holds (an edge of 64, 32768
    points, 64 ions) match the context path, and each input the path does
    not take is rejected before any device work: 65 ions, a sheared cell,
    a non-positive charge, a non-finite position."""
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    d = inputs.hydrogen(64, 1.0, 5.0e4, 8, seed=17, functional="vt84f")
    for fn, grid in [("vt84f", (64, 64, 8)), ("fttf", (8, 64, 64)), ("sga", (32, 32, 32))]:
        N = int(np.prod(grid))
        rng = np.random.default_rng(N + len(fn))
        phi = np.sqrt(64.0 / np.prod(d["L"])) * (1.0 + 0.1 * rng.standard_normal(N))
        with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], fn) as ctx:
            E_ref, v_ref = ctx.energy_potential(phi)
        phi_d = torch.tensor(phi, dtype=torch.float64, device="cuda")
        v_d = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        E = ofdft.ofdft_energy_potential_static(np.diag(d["L"]), grid, d["ions"], d["Z"], d["T"], fn,
                                                phi_d.data_ptr(), v_d.data_ptr())
        v = v_d.cpu().numpy().reshape(grid)
        for k in ("F_tot", "F_s", "E_H", "E_loc", "F_xc", "E_ion", "P"):
            assert abs(E[k] - E_ref[k]) <= 1e-10 * max(abs(E_ref["F_tot"]), 1.0), (fn, grid, k)
        assert np.max(np.abs(v - v_ref)) <= 1e-9 * np.max(np.abs(v_ref)), (fn, grid)
    buf = torch.zeros(16 ** 3, dtype=torch.float64, device="cuda")
    ions65 = np.vstack([d["ions"], d["ions"][:1] + 0.3])
    sheared = np.diag(d["L"]) + np.array([[0.0, 0.0, 0.0], [0.4, 0.0, 0.0], [0.0, 0.0, 0.0]])
    bad_Z = d["Z"].copy()
    bad_Z[3] = 0.0
    bad_pos = d["ions"].copy()
    bad_pos[5, 1] = np.nan
    for cell, ions, Z in [(np.diag(d["L"]), ions65, np.ones(65)), (sheared, d["ions"], d["Z"]),
                          (np.diag(d["L"]), d["ions"], bad_Z), (np.diag(d["L"]), bad_pos, d["Z"])]:
        with pytest.raises(ofdft.OfdftError) as e:
            ofdft.ofdft_energy_potential_static(cell, (16, 16, 16), ions, Z, d["T"], "fttf",
                                                buf.data_ptr(), buf.data_ptr())
        assert e.value.status == -1


def test_static_entry_point_refuses_a_capturing_stream():
    """The call copies from pageable host memory and synchronises, which a
    stream capture cannot hold: on a capturing stream it returns
    OFDFT_EINVAL before any work, and the capture stays valid."""
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    cfg = inputs.config_single_point()
    grid = (16, 16, 16)
    buf = torch.ones(16 ** 3, dtype=torch.float64, device="cuda")
    x = torch.zeros(1, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(g, stream=s):
        x += 1.0
        try:
            ofdft.ofdft_energy_potential_static(np.diag(cfg["L"]), grid, cfg["ions"], cfg["Z"], cfg["T"],
                                                "fttf", buf.data_ptr(), buf.data_ptr(), stream=s.cuda_stream)
        except ofdft.OfdftError as e:
            status = e.status
    assert status == -1
    g.replay()
    torch.cuda.synchronize()
    assert float(x.item()) == 1.0
