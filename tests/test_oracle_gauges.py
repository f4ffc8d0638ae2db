"""Pins of the oracle's gauge levels (the water level at wave gauges, the
adjoint workload's loss): closed forms on hand-made surfaces.

  * a flat surface at H + c reads c at every gauge covered by it;
  * a gauge farther than 2 l from every surface particle reads 0, and only
    free-surface fluid particles count (interior particles and walls at other
    heights change nothing);
  * on a regular row of surface particles, a linear surface z = H + a (x - x_g)
    reads 0 at a gauge on a particle (the weights are symmetric there), and
    opposite levels at gauges b to either side of it (mirror images).
"""
import numpy as np

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S


def _row(n=41, d0=0.01, H=0.2):
    sc = S.small_tank(dim=2, kind="E", L=0.5, H=H, d0=d0, jitter=0.0, bathy=S.Bathymetry())
    x = np.arange(n) * d0
    sc.x, sc.z = x.copy(), np.full(n, H)
    for k in ("y", "u", "v", "w", "p", "jbar"):
        setattr(sc, k, np.zeros(n))
    sc.type = np.zeros(n, dtype=np.int32)
    return sc


def test_flat_surface_reads_its_height():
    sc = _row()
    fs = np.ones(sc.n, dtype=np.int32)
    z = sc.z + 0.013
    eta = O.gauge_levels(sc, fs, [0.1, 0.203, 0.35], z=z)
    assert np.allclose(eta, 0.013, rtol=0, atol=1e-15)


def test_only_surface_fluid_particles_count_and_far_gauges_read_zero():
    sc = _row()
    fs = np.ones(sc.n, dtype=np.int32)
    z = sc.z.copy()
    fs[:10] = 0
    z[:10] += 5.0                       # interior particles far off the surface
    sc.type[10:14] = 1                  # walls at another height
    z[10:14] -= 3.0
    l, _, _ = O.radii(sc)
    eta = O.gauge_levels(sc, fs, [0.3, 0.40 + 2.0 * l + 1e-9], z=z)
    assert abs(eta[0]) < 1e-15
    assert eta[1] == 0.0


def test_linear_surface_on_a_regular_row():
    sc = _row()
    fs = np.ones(sc.n, dtype=np.int32)
    a, xg = 0.05, 0.2
    z = sc.params["H"] + a * (sc.x - xg)
    eta = O.gauge_levels(sc, fs, [xg], z=z)
    assert abs(eta[0]) < 1e-15          # symmetric weights about a particle
    up, down = O.gauge_levels(sc, fs, [xg + 0.004, xg - 0.004], z=z)
    assert abs(up + down) < 1e-15       # mirror images about the particle at x_g
    assert 0.0 < up < a * 0.004 * 1.5   # the right sign, near a b
