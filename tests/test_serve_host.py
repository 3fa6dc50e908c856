"""Host logic of the serving loop (ofdft_serve_*) in dry-run mode: admission
in arrival order while a slot is free and the footprint fits the budget,
budget and slot limits never exceeded, oversize requests refused.  No GPU
work runs (each request only sleeps)."""
import numpy as np
import pytest

from paper_1406_0835_gb300 import ofdft


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _req(server, grid, nat=8):
    ions = np.random.default_rng(nat).uniform(0, 5.0, (nat, 3))
    return server.submit((5.0, 5.0, 5.0), grid, ions, np.ones(nat), 1e5, "vt84f", "fp64", md_steps=1)


def test_footprint_grows_with_grid_and_precision():
    a = ofdft.ofdft_footprint((32, 32, 32), 8, "fp64")
    b = ofdft.ofdft_footprint((64, 64, 64), 8, "fp64")
    c = ofdft.ofdft_footprint((64, 64, 64), 8, "mixed")
    assert 0 < a < b < c
    # FP64 fields: at least nine real fields and four half spectra of N doubles
    assert b > (9 + 4) * 64 ** 3 * 8
    assert ofdft.ofdft_footprint((30, 32, 32), 8, "fp64") > 0      # 30 = 2 3 5
    with pytest.raises(ofdft.OfdftError):
        ofdft.ofdft_footprint((31, 32, 32), 8, "fp64")


def test_footprint_counts_the_per_ion_tables():
    """Per ion a context holds its axis phase tables (binary64, nx + ny +
    nz/2 + 1 complex values) and their double-float copies (x, y and z
    ions-fastest, z per ion), plus force partials: growing the ion count
    at fixed grid grows the footprint by at least that much."""
    nx, ny, nz = 96, 96, 96
    K = nz // 2 + 1
    a = ofdft.ofdft_footprint((nx, ny, nz), 128, "fp64")
    b = ofdft.ofdft_footprint((nx, ny, nz), 1024, "fp64")
    tables = (1024 - 128) * (2 * nx + 2 * ny + 3 * K) * 16
    assert b - a >= tables


def test_admission_order_budget_and_slots():
    small = ofdft.ofdft_footprint((32, 32, 32), 8, "fp64")
    big = ofdft.ofdft_footprint((64, 64, 64), 8, "fp64")
    budget = big + 1.5 * small          # the big one and one small, never two small beside it
    with ofdft.Server(max_slots=3, hbm_budget_bytes=budget, dry_run_ms=60, max_bypass=0) as s:
        ids = [_req(s, (64, 64, 64)), _req(s, (32, 32, 32)), _req(s, (32, 32, 32)),
               _req(s, (32, 32, 32)), _req(s, (64, 64, 64))]
        assert s.poll(ids[-1]) is None or s.poll(ids[-1])["status"] == 0
        s.drain(timeout_s=30.0)
        res = [s.poll(i) for i in ids]
        peak_bytes, peak_running = s.peaks()
    assert all(r["status"] == 0 and r["steps_done"] == 1 for r in res)
    assert peak_bytes <= budget
    assert 2 <= peak_running <= 3                  # requests overlapped, never beyond the slots
    admits = [r["t_admit"] for r in res]
    assert admits == sorted(admits)                # first come, first admitted
    for r in res:
        assert r["t_submit"] <= r["t_admit"] < r["t_done"]
    # the last big request had to wait for the first one's memory, and for
    # all but one small request's (only then do big + small fit)
    assert res[4]["t_admit"] >= res[0]["t_done"] - 1e-3
    assert res[4]["t_admit"] >= min(res[2]["t_done"], res[3]["t_done"]) - 1e-3


def test_smaller_requests_pass_a_waiting_one_a_bounded_number_of_times():
    """A big request that does not fit yet is passed by later small ones
    that do, at most max_bypass of them; the next small one waits behind it,
    so the big one is not starved."""
    small = ofdft.ofdft_footprint((32, 32, 32), 8, "fp64")
    big = ofdft.ofdft_footprint((96, 96, 96), 8, "fp64")
    budget = big + 3.5 * small        # beside a big one: three small (memory), never a second big
    assert 2 * big > budget
    with ofdft.Server(max_slots=5, hbm_budget_bytes=budget, dry_run_ms=150, max_bypass=2) as s:
        ids = [_req(s, (96, 96, 96)), _req(s, (96, 96, 96)), _req(s, (32, 32, 32)),
               _req(s, (32, 32, 32)), _req(s, (32, 32, 32))]
        s.drain(timeout_s=30.0)
        A, B, C, D, E = [s.poll(i) for i in ids]
        peak_bytes, _ = s.peaks()
    assert all(r["status"] == 0 for r in (A, B, C, D, E))
    assert peak_bytes <= budget
    assert C["t_admit"] < B["t_admit"] and D["t_admit"] < B["t_admit"]   # passed the waiting big one
    assert B["t_admit"] >= A["t_done"] - 1e-3                           # it waited for memory
    assert E["t_admit"] >= B["t_admit"]                                 # the third could not pass it


def test_oversize_and_bad_requests_are_refused():
    small = ofdft.ofdft_footprint((32, 32, 32), 8, "fp64")
    with ofdft.Server(max_slots=1, hbm_budget_bytes=2 * small, dry_run_ms=1) as s:
        with pytest.raises(ofdft.OfdftError) as e:
            _req(s, (128, 128, 128))
        assert e.value.status == -2
        with pytest.raises(ofdft.OfdftError) as e:
            _req(s, (33, 32, 32))
        assert e.value.status == -1
        with pytest.raises(ofdft.OfdftError):
            s.poll(12345)                          # never submitted


def test_dry_run_needs_a_budget():
    with pytest.raises(ofdft.OfdftError):
        ofdft.Server(max_slots=1, hbm_budget_bytes=0.0, dry_run_ms=1)
    with pytest.raises(ofdft.OfdftError):
        ofdft.Server(max_slots=1, hbm_budget_bytes=1e9, dry_run_ms=1, max_bypass=-1)


def _req_steps(server, grid, md_steps, nat=8):
    ions = np.random.default_rng(nat).uniform(0, 5.0, (nat, 3))
    return server.submit((5.0, 5.0, 5.0), grid, ions, np.ones(nat), 1e5, "vt84f", "fp64", md_steps=md_steps)


def test_cancel_queued_running_finished_and_unknown_requests():
    """A queued request cancels at once (status OFDFT_ECANCELED, no steps,
    never admitted) and frees its place for the one behind it; a running
    one stops before its next MD step with the steps it completed; a
    finished one keeps its result; an unknown id is an error."""
    small = ofdft.ofdft_footprint((32, 32, 32), 8, "fp64")
    with ofdft.Server(max_slots=1, hbm_budget_bytes=4 * small, dry_run_ms=400, max_bypass=0) as s:
        run = _req_steps(s, (32, 32, 32), 10)       # admitted at once: 11 parts of ~36 ms
        queued = _req_steps(s, (32, 32, 32), 2)     # waits for the only slot
        after = _req_steps(s, (32, 32, 32), 0)
        t0 = s.clock()
        while s.clock() - t0 < 0.12:                 # let the first run a few of its steps
            pass
        s.cancel(queued)
        r_q = s.poll(queued)
        assert r_q is not None and r_q["status"] == -8 and r_q["steps_done"] == 0 and r_q["t_admit"] == -1.0
        s.cancel(run)
        s.drain(timeout_s=30.0)
        r_run, r_after = s.poll(run), s.poll(after)
        s.cancel(after)                              # finished: no effect
        assert s.poll(after) == r_after
        with pytest.raises(ofdft.OfdftError) as e:
            s.cancel(10 ** 9)
        assert e.value.status == -1
    assert r_run["status"] == -8 and 1 <= r_run["steps_done"] < 10
    assert r_run["t_done"] - r_run["t_admit"] < 0.35     # stopped well before its 400 ms
    assert r_after["status"] == 0
    assert r_after["t_admit"] >= r_run["t_done"] - 1e-3   # the cancelled queued one did not hold the slot
