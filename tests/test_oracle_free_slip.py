"""Pins of the oracle's free-slip walls (Sec. 3.5): a wall particle carries
v = (I - 2 n (x) n) v_wall, with v_wall the SPH interpolation of the fluid
velocity at the wall particle and n the outer unit normal in physical space.

  * a uniform flow parallel to a sloped bottom (BF map, slope 0.15) is carried
    unchanged by the bottom wall particles (away from the corners), so the
    near-wall fluid sees a uniform field: the viscous term vanishes and
    v* = v + dt g exactly, while under no-slip it does not;
  * a uniform flow INTO the sloped bottom (along -n) is reflected: the bottom
    wall particles carry +U n, so the physical normal is the slope's normal
    (h_x, -1)/sqrt(1 + h_x^2), not the projected (0, -1);
  * no-slip walls carry zero.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

SLOPE = 0.15


def _tank(u, w, slip):
    bathy = S.Bathymetry(h0=0.01, slope_x=SLOPE)
    prm = dict(d0=0.01, H=0.18, H_hat=0.18, nu_k=1.0e-2, smagorinsky=0, gamma_over_dt=0.0,
               wall_slip=slip)
    sc = S.build_tank("pin_slip", 2, "BF", 1.0, bathy, prm, 0.5, jitter=0.1, seed=3)
    f = sc.type == S.FLUID
    sc.u[f] = u
    sc.w[f] = w
    return sc


def _bottom_walls_away_from_corners(sc, margin):
    wall = sc.type == S.WALL
    bottom = wall & (np.abs(sc.z - (0.01 + SLOPE * sc.x)) < 1e-12)
    return bottom & (sc.x > margin) & (sc.x < 0.5 - margin)


def test_tangential_flow_passes_free_slip_walls_unchanged():
    n = np.array([SLOPE, -1.0]) / np.hypot(SLOPE, 1.0)
    t = np.array([1.0, SLOPE]) / np.hypot(SLOPE, 1.0)
    U = 0.3
    sc = _tank(U * t[0], U * t[1], 1)
    _, info = O.step(sc, probe=True)
    assert info["rc"] == 0
    _, re, re2 = O.radii(sc)
    bw = _bottom_walls_away_from_corners(sc, 3 * re)
    assert bw.sum() > 20
    assert np.allclose(info["vwall"][0, bw], U * t[0], rtol=0, atol=1e-12)
    assert np.allclose(info["vwall"][1, bw], U * t[1], rtol=0, atol=1e-12)
    # fluid rows next to those walls, seeing no other wall particle
    xh, _ = O.projected(sc)
    row, col = O.neighbours(2, xh, re, re2)
    wall = sc.type == S.WALL
    rows = [i for i in np.flatnonzero(sc.type == S.FLUID)
            if np.any(bw[col[row[i]:row[i + 1]]]) and
            np.all(~wall[col[row[i]:row[i + 1]]] | bw[col[row[i]:row[i + 1]]])]
    rows = np.array(rows)
    assert rows.size > 10
    dt, g = sc.params["dt"], sc.params["g"]
    acc_u = (info["vstar"][0, rows] - sc.u[rows]) / dt
    acc_w = (info["vstar"][1, rows] - sc.w[rows]) / dt + g
    assert np.abs(acc_u).max() < 1e-9 and np.abs(acc_w).max() < 1e-9
    # no-slip: the walls carry zero, the same rows feel the wall's shear
    sc0 = _tank(U * t[0], U * t[1], 0)
    _, info0 = O.step(sc0, probe=True)
    assert np.abs(info0["vwall"]).max() == 0.0
    acc0 = (info0["vstar"][0, rows] - sc0.u[rows]) / dt
    assert np.abs(acc0).max() > 1.0


def test_normal_flow_is_reflected_about_the_slope_normal():
    n = np.array([SLOPE, -1.0]) / np.hypot(SLOPE, 1.0)
    U = 0.2
    sc = _tank(U * n[0], U * n[1], 1)          # flowing into the bottom
    _, info = O.step(sc, probe=True)
    _, re, _ = O.radii(sc)
    bw = _bottom_walls_away_from_corners(sc, 3 * re)
    assert np.allclose(info["vwall"][0, bw], -U * n[0], rtol=0, atol=1e-12)
    assert np.allclose(info["vwall"][1, bw], -U * n[1], rtol=0, atol=1e-12)
