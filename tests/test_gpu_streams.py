"""The three-stream GGA evaluation (the Hartree chain beside the gradient
chain, the derivative passes in pairs, joined before the final z pass)
changes only when kernels run, not what they compute: a minimisation
driven by the CUDA graph with its parallel branches and the same
minimisation with every kernel on one stream (host-driven loops, which a
selected kernel timer forces) give bit-identical densities, energies and
iteration counts, for FP64 and mixed-precision contexts."""
import numpy as np
import pytest

from paper_1406_0835_gb300 import inputs, ofdft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_forked_and_single_stream_evaluations_agree_bit_for_bit(precision):
    d = inputs.hydrogen(16, 1.0, 3.125e4, 24, seed=4, functional="vt84f")
    grid = (24, 24, 24)
    out = []
    for single_stream in (False, True):
        with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], "vt84f", precision=precision) as ctx:
            if single_stream:
                ofdft.ofdft_timer_select(ctx.ctx, "pw")
            E, st = ctx.minimize(gtol=1e-9)
            n = ctx.density()
        out.append((E, st, n))
    (E0, s0, n0), (E1, s1, n1) = out
    assert s0["iterations"] == s1["iterations"] and s0["evaluations"] == s1["evaluations"]
    assert E0["F_tot"] == E1["F_tot"] and E0["P"] == E1["P"]
    assert np.array_equal(n0, n1)
