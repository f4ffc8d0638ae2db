"""Checkpointed forward run and segment replay (vct.Checkpointer, with
vct_reset_history at every checkpoint): the run ends in the same state as the
same steps queued one by one with the same resets, and a replayed segment
reproduces that run's states bit for bit (the reverse sweep of an adjoint
recomputes each segment from its checkpoint)."""
import numpy as np
import pytest

from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_replay_reproduces_the_forward_run(precision):
    from paper_2607_28872_b300 import vct as V
    sc = S.small_tank(dim=2, kind="SIGMA", L=0.3, H=0.1, d0=0.01, seed=8, with_wave=True,
                      precision=precision)
    every, nsteps = 2, 5   # the tank stays well-posed for these few steps
    s_ref = V.Solver(sc)
    st = V.DeviceState(sc)
    ref = []
    for step in range(nsteps):
        if step % every == 0:
            s_ref.vct_reset_history()
        s_ref.vct_step(st, 1)
        ref.append(st.numpy())
    solver = V.Solver(sc)
    cp = V.Checkpointer(solver, every=every)
    state = V.DeviceState(sc)
    cp.run(state, nsteps)
    assert cp.lengths == [2, 2, 1] and len(cp.snapshots) == 3
    end = state.numpy()
    for k in ("x", "z", "u", "w", "p", "jbar"):
        assert np.array_equal(end[k], ref[-1][k]), k
    for seg, first in ((1, 2), (2, 4), (0, 0)):
        states = cp.replay(seg)
        assert len(states) == cp.lengths[seg]
        for q, sq in enumerate(states):
            g = sq.numpy()
            for k in ("x", "z", "u", "w", "p", "jbar"):
                assert np.array_equal(g[k], ref[first + q][k]), (seg, q, k)
