"""The gauge loss of the adjoint workload on the GPU (vct_gauge_loss): the water
level at wave gauges (Sec. 4.4.2) from the free-surface particles, its squared
sum and the gradient with respect to the particle positions.

  * levels and loss against the oracle's definition (oracle.gauge_levels) on
    the 2-D wave (eight gauges, one on the crest) and a 3-D BFE tank with a
    wave (four gauges in x and y), flags from the oracle's step;
  * the gradient against central differences of the oracle's loss at every
    particle with a non-zero gradient component (and zero elsewhere);
  * bad gauge counts are rejected.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


def _case(dim):
    if dim == 2:
        sc = S.solitary_sigma(precision=0)
        gauges = np.linspace(2.0, 8.0, 8)
    else:
        sc = S.small_tank(dim=3, kind="BFE", L=0.3, W=0.12, H=0.06, d0=0.01, seed=4, aspect=2.0,
                          with_wave=True)
        gauges = np.array([[0.05, 0.03], [0.11, 0.06], [0.17, 0.05], [0.26, 0.09]])
    _, info = O.step(sc, probe=True, max_iter=1)
    return sc, gauges, info["fs"].astype(np.int32)


@pytest.mark.parametrize("dim", [2, 3])
def test_gauge_loss_and_gradient(dim):
    import torch
    from paper_2607_28872_b300 import vct as V
    sc, gauges, fs = _case(dim)
    s = V.Solver(sc)
    st = V.DeviceState(sc)
    loss, eta, grad = s.vct_gauge_loss(st, torch.tensor(fs, device="cuda"), gauges)
    grad = grad.cpu().numpy()
    eta_o = O.gauge_levels(sc, fs, gauges)
    loss_o = O.gauge_loss(sc, fs, gauges)
    assert np.abs(eta).max() > 1e-3                     # the wave reaches a gauge
    assert np.abs(eta - eta_o).max() <= 1e-12 * np.abs(eta_o).max()
    assert abs(loss - loss_o) <= 1e-12 * loss_o
    y0 = sc.y if sc.dim == 3 else None
    coords = dict(x=sc.x.copy(), y=None if y0 is None else y0.copy(), z=sc.z.copy())
    axes = ("x", "z") if dim == 2 else ("x", "y", "z")
    nz = np.flatnonzero(np.abs(grad).max(axis=0) > 0)
    assert nz.size > 10
    assert np.all(fs[nz] == 1)                           # only surface particles count
    rng = np.random.default_rng(3)
    pick = rng.choice(nz, size=min(60, nz.size), replace=False)
    h = 1e-7
    worst = 0.0
    for i in pick:
        for k, a in enumerate(axes):
            cp = {q: (None if v is None else v.copy()) for q, v in coords.items()}
            cm = {q: (None if v is None else v.copy()) for q, v in coords.items()}
            cp[a][i] += h
            cm[a][i] -= h
            fd = (O.gauge_loss(sc, fs, gauges, **cp) - O.gauge_loss(sc, fs, gauges, **cm)) / (2 * h)
            scale = np.abs(grad).max()
            worst = max(worst, abs(fd - grad[k, i]) / scale)
    print(f"PARITY gauge loss {dim}-D: loss {loss:.6e}, gradient err {worst:.2e} at {pick.size} particles")
    assert worst < 1e-6


def test_gauge_counts_are_validated():
    import torch
    from paper_2607_28872_b300 import vct as V
    sc, _, fs = _case(2)
    s = V.Solver(sc)
    st = V.DeviceState(sc)
    f = torch.tensor(fs, device="cuda")
    for bad in (np.zeros(0), np.linspace(0.0, 1.0, 17), np.array([np.nan])):
        with pytest.raises(V.VCTError) as e:
            s.vct_gauge_loss(st, f, bad)
        assert e.value.status == V.VCT_ERR_ARG
