"""Failure detection without faulting the GPU.

  * bounded waits: the pressure solve's grid barriers poll at most
    spin_limit times; with a limit of one poll the blocks cannot all meet,
    every wait gives up, the kernel ends and the call returns
    VCT_ERR_TIMEOUT with the caller's state untouched; a context with the
    default limit then steps the same state normally;
  * an isolated fluid particle (no neighbours) is not an error: it falls
    under gravity alone (the oracle alike);
  * a singular SPH(2) moment matrix at a particle off the free surface is:
    the step reports VCT_ERR_SINGULAR naming that particle and the caller's
    state is untouched (the oracle reports the same).
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


def test_isolated_particle_falls_freely():
    """A fluid particle without neighbours (a splash) is isolated: flagged 2,
    no corrected derivatives, no pressure; it falls under gravity alone while
    the rest of the tank steps normally (the oracle alike)."""
    from paper_2607_28872_b300 import vct as V
    sc = _tank()
    f = np.flatnonzero(sc.type == S.FLUID)
    k = int(f[len(f) // 2])
    sc.x[k] = 0.3
    sc.z[k] = 0.3                                  # far above the water, inside the box
    assert sc.box_hi[2] > 0.3
    ost, info = O.step(sc, probe=True)
    assert info["rc"] == 0 and info["fs"][k] == 2
    s = V.Solver(sc)
    st = V.DeviceState(sc)
    out, _ = s.vct_step_probe(st)
    g = st.numpy()
    assert int(out["fs"].cpu().numpy()[k]) == 2
    dt, grav = sc.params["dt"], sc.params["g"]
    assert abs(g["w"][k] - (sc.w[k] - grav * dt)) < 1e-12
    assert abs(g["u"][k] - sc.u[k]) < 1e-12 and g["p"][k] == 0.0
    assert abs(g["w"][k] - ost.w[k]) < 1e-12


def _cross():
    """A fluid particle whose neighbours lie on two lines through it (x and z
    axes, two on each side): its correction matrix is regular but the cross
    moment x z vanishes for every neighbour, so the SPH(2) moment matrix M_i
    is singular, at a particle that is not on the free surface."""
    sc = S.small_tank(dim=2, kind="E", L=0.1, H=0.05, d0=0.01, jitter=0.0, aspect=1.0,
                      bathy=S.Bathymetry())
    d0 = 0.01
    pts = [(0.0, 0.0)] + [(sg * k * d0, 0.0) for sg in (-1, 1) for k in (1, 2)] + \
          [(0.0, sg * k * d0) for sg in (-1, 1) for k in (1, 2)]
    pts = np.array(pts) + 0.5
    n = len(pts)
    for key in ("y", "u", "v", "w", "p", "jbar"):
        setattr(sc, key, np.zeros(n))
    sc.x, sc.z = pts[:, 0].copy(), pts[:, 1].copy()
    sc.type = np.zeros(n, dtype=np.int32)
    sc.box_lo, sc.box_hi = (0.0, 0.0, 0.0), (1.0, 0.0, 1.0)
    return sc


def test_singular_moment_matrix_is_reported():
    from paper_2607_28872_b300 import vct as V
    sc = _cross()
    _, info = O.step(sc, max_iter=5)
    assert info["rc"] == 3                          # the oracle's singular code
    st = V.DeviceState(sc)
    before = st.numpy()
    s = V.Solver(sc)
    with pytest.raises(V.VCTError) as e:
        s.vct_step(st, 1)
    assert e.value.status == V.VCT_ERR_SINGULAR
    assert 0 <= e.value.particle < sc.n           # the first offender of the crafted set
    after = st.numpy()
    for key in ("x", "z", "u", "w", "p"):
        assert np.array_equal(before[key], after[key]), key
