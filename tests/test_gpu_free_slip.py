"""Free-slip walls (Sec. 3.5) and the 3-D sigma dam break (Sec. 4.4.3) on the GPU.

  * the wall particles' velocities (probe output) against the oracle's, and
    one step through vct_step_probe against the oracle's step with free-slip
    walls (2-D BF over a slope, 2-D sigma with a wave, 3-D BFE);
  * a coarse copy of the dam break (d0 = 1 cm) against the oracle, one step;
  * the dam break at its stated resolution (d0 = 0.25 cm, 98k fluid
    particles, dt = 1e-4 s) for 150 steps: the water column starts to
    collapse into the dry part of the basin, the state stays bounded and the
    total volume (sum of V0 / Jbar, Condition C) stays within 1 %.  (Near
    step 190 a free-surface particle at the upper corner of the column and the
    left wall is ejected and the run breaks down; the horizon is stated.)
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

from test_gpu_parity import _probe_compare, rel, report

pytestmark = pytest.mark.gpu

CASES = [
    ("bf2d_slope", lambda: S.small_tank(dim=2, kind="BF", L=0.37, H=0.1, d0=0.01, seed=1,
                                        bathy=S.Bathymetry(h0=-0.02, slope_x=0.1), with_wave=True)),
    ("sigma2d_wave", lambda: S.small_tank(dim=2, kind="SIGMA", L=0.41, H=0.1, d0=0.01, seed=2,
                                          with_wave=True)),
    ("bfe3d", lambda: S.small_tank(dim=3, kind="BFE", L=0.17, W=0.09, H=0.06, d0=0.01, seed=4,
                                   aspect=2.0, with_wave=True)),
]


@pytest.fixture(scope="module")
def vct():
    from paper_2607_28872_b300 import vct as V
    V.load_library()
    return V


@pytest.mark.parametrize("precision,tol,band", [(0, 1e-12, 1e-9), (1, 1e-5, 1e-5)],
                         ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_free_slip_step_parity(vct, name, make, precision, tol, band):
    sc = make()
    sc.params["wall_slip"] = 1
    # the wall velocities themselves (FP64 in both forms)
    s2 = sc.copy()
    s2.params["precision"] = precision
    solver = vct.Solver(s2)
    out, _ = solver.vct_step_probe(vct.DeviceState(s2))
    _, info = O.step(s2, probe=True, max_iter=1)
    wall = sc.type == S.WALL
    assert np.abs(info["vwall"][:, wall]).max() > 1e-3
    # FP64 in both forms, from the particle volumes V0 J/Jbar (Jbar of the sigma
    # smoothing comes from FP32 pair distances in the mixed form)
    assert report(f"slip {name} p{precision} vwall",
                  rel(out["vwall"].cpu().numpy()[:, wall], info["vwall"][:, wall]), tol)
    _probe_compare(vct, sc, precision, tol, band, "slip-" + name)


@pytest.mark.parametrize("precision,tol,band", [(0, 1e-12, 1e-9), (1, 1e-5, 1e-5)],
                         ids=["fp64", "mixed"])
def test_dam_break_coarse_parity(vct, precision, tol, band):
    sc = S.dam_break_sigma_3d(d0=0.01)
    _probe_compare(vct, sc, precision, tol, band, "dam-break-coarse")


def test_dam_break_full_resolution_runs():
    from paper_2607_28872_b300 import vct as V
    sc = S.dam_break_sigma_3d()
    assert sc.n_fluid > 90_000
    f = sc.type == S.FLUID
    s = V.Solver(sc)
    st = V.DeviceState(sc)
    s.vct_step(st, 1)
    v0 = np.sum(sc.params["d0"] ** 3 / st.numpy()["jbar"][f])
    x0 = sc.x[f].max()
    s.vct_step(st, 149)
    g = st.numpy()
    assert np.all(np.isfinite(g["x"][f])) and np.all(np.isfinite(g["p"][f]))
    vmax = np.sqrt(g["u"] ** 2 + g["v"] ** 2 + g["w"] ** 2)[f].max()
    assert vmax < 2.0 * np.sqrt(sc.params["g"] * sc.params["H"])
    e_v = np.sum(sc.params["d0"] ** 3 / g["jbar"][f]) / v0 - 1.0
    front = g["x"][f].max()
    print(f"PARITY dam break 150 steps: e_V={e_v:.3e} front {x0:.3f} -> {front:.3f} m, "
          f"max |v| {np.sqrt(g['u'] ** 2 + g['v'] ** 2 + g['w'] ** 2)[f].max():.3f} m/s")
    assert abs(e_v) < 1e-2
    assert front > x0 + 0.001                     # the column has started to collapse
