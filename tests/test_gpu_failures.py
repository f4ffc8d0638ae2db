"""Failure detection without faulting the GPU.

  * bounded waits: the pressure solve's grid barriers poll at most
    spin_limit times; with a limit of one poll the blocks cannot all meet,
    every wait gives up, the kernel ends and the call returns
    VCT_ERR_TIMEOUT with the caller's state untouched; a context with the
    default limit then steps the same state normally;
  * a singular moment matrix: a fluid particle with no neighbours has
    B_i = 0, the step reports VCT_ERR_SINGULAR naming that particle, and the
    caller's state is untouched (the oracle reports the same).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


def _tank():
    return S.small_tank(dim=2, kind="SIGMA", L=0.6, H=0.12, d0=0.01, seed=4, with_wave=True)


def test_barrier_wait_runs_out():
    from paper_2607_28872_b300 import vct as V
    sc = _tank()
    st = V.DeviceState(sc)
    before = st.numpy()
    s = V.Solver(sc, spin_limit=1)
    with pytest.raises(V.VCTError) as e:
        s.vct_step(st, 1)
    assert e.value.status == V.VCT_ERR_TIMEOUT
    after = st.numpy()
    for k in ("x", "z", "u", "w", "p", "jbar"):
        assert np.array_equal(before[k], after[k]), k
    s.close()
    ok = V.Solver(sc)
    stats = ok.vct_step(st, 2)
    assert stats.steps_done == 2 and stats.krylov_iters_total > 0


def test_isolated_particle_is_singular():
    from paper_2607_28872_b300 import vct as V
    sc = _tank()
    f = np.flatnonzero(sc.type == S.FLUID)
    k = int(f[len(f) // 2])
    sc.x[k] = 0.3
    sc.z[k] = 0.3                                  # far above the water, inside the box
    assert sc.box_hi[2] > 0.3
    _, info = O.step(sc)
    assert info["rc"] == 3                          # the oracle's singular code
    st = V.DeviceState(sc)
    before = st.numpy()
    s = V.Solver(sc)
    with pytest.raises(V.VCTError) as e:
        s.vct_step(st, 1)
    assert e.value.status == V.VCT_ERR_SINGULAR
    assert e.value.particle == k
    after = st.numpy()
    for key in ("x", "z", "u", "w", "p"):
        assert np.array_equal(before[key], after[key]), key
