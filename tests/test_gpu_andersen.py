"""GPU parity of NVT MD with Andersen collisions (the thermostat of the
paper's MD runs, Sec. VI): velocity-Verlet steps without Nose-Hoover, each
followed by a round of collisions with the same random numbers on both sides.
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


def test_andersen_md_matches_oracle():
    d = inputs.hydrogen(8, 1.0, 3.125e4, 16, seed=2, functional="sga", vel_seed=3)
    grid = (16, 16, 16)
    so = O.System(d["L"], grid, d["ions"], d["Z"], d["T"], "sga")
    st = O.MDState(d["ions"], d["vel"], d["masses"], d["T"], dt_fs=0.2)
    O.md_prepare(so, st, gtol=1e-10)
    prob = 0.4
    with ofdft.Context(d["L"], grid, d["ions"], d["Z"], d["T"], "sga") as ctx:
        ctx.md_step(0.2, 0.0, nsteps=0, pos=d["ions"], vel=d["vel"], gtol=1e-10)
        for step in range(3):
            O.md_step(so, st, gtol=1e-10, thermostat=False)
            ctx.md_step(0.2, 0.0, nsteps=1, gtol=1e-10)
            u, xi = inputs.andersen_draws(8, seed=100 + step)
            n_o = O.md_andersen(st, d["T"], prob, u, xi)
            assert ctx.md_andersen(d["T"], prob, u, xi) == n_o
            _, vel = ctx.md_state()
            hit = u < prob
            # redrawn velocities: the same correctly rounded arithmetic on both sides
            np.testing.assert_allclose(vel[hit], st.V[hit], rtol=1e-15, atol=0)
        pos, vel = ctx.md_state()
        np.testing.assert_allclose(pos, st.R, rtol=0, atol=1e-10)
        np.testing.assert_allclose(vel, st.V, rtol=0, atol=1e-12)
        with pytest.raises(ofdft.OfdftError):
            ctx.md_andersen(d["T"], 1.5, u, xi)
        with pytest.raises(ofdft.OfdftError):
            ctx.md_andersen(-1.0, 0.5, u, xi)
