"""Pins of the oracle's particle regularisation (dynamic stabilization, XSPH on
free-surface particles, optimized particle shifting; Sec. 4.1 gives their
parameters, the formulas are restated from the cited methods).

Each pin is a property the methods fix, not a retyped formula:
  * dynamic stabilization restores the allowed distance d_DS exactly for an
    isolated pair (half each for two fluid particles, all of it against a
    wall), keeps the pair's momentum, acts in projected space (a stretched
    map changes the physical displacement by 1/alpha) and leaves pairs beyond
    d_DS alone;
  * shifting is zero on a symmetric lattice and for particles at rest, moves
    a displaced particle back towards its lattice site, and moves free-surface
    particles of a flat surface only along the surface (the normal of Marrone
    et al., from the renormalisation matrix);
  * XSPH leaves a uniform velocity field unchanged, touches only free-surface
    particles and reduces the relative velocity of a pair;
  * with every parameter at zero the state is untouched.
"""
import numpy as np

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

D0 = 0.01
DT = 1.0e-3


def make(xs, zs, types=None, u=None, w=None, kind="E", aspect=1.0, **prm):
    """A 2-D scenario with the given particles (physical positions)."""
    n = len(xs)
    params = dict(S.DEFAULT_PARAMS)
    params.update(d0=D0, dt=DT, H=1.0, H_hat=aspect, smagorinsky=0)
    params.update(prm)
    t = np.zeros(n, np.int32) if types is None else np.asarray(types, np.int32)
    z = np.zeros(n)
    return S.Scenario(name="pin", dim=2, map_kind=kind, aspect=aspect, bathy=S.Bathymetry(),
                      params=params, x=np.asarray(xs, float), y=z.copy(),
                      z=np.asarray(zs, float), u=np.zeros(n) if u is None else np.asarray(u, float),
                      v=z.copy(), w=np.zeros(n) if w is None else np.asarray(w, float),
                      p=z.copy(), jbar=np.ones(n) * aspect, type=t,
                      box_lo=(-1.0, 0.0, -1.0), box_hi=(2.0, 0.0, 2.0))


def run(sc, fs=None, **over):
    st = O.OracleState(sc)
    O.regularise(sc, st, fs=fs, **over)
    return st


def test_all_off_is_identity():
    rng = np.random.default_rng(0)
    sc = make(rng.uniform(0, 0.05, 40), rng.uniform(0, 0.05, 40), u=rng.normal(size=40),
              w=rng.normal(size=40))
    st = run(sc, fs=np.ones(40, np.int32))
    for k in ("x", "z", "u", "w"):
        assert np.array_equal(getattr(st, k), getattr(sc, k))


def test_ds_restores_allowed_distance_fluid_pair():
    r0 = 0.3 * D0
    sc = make([0.0, r0], [0.0, 0.0], u=[0.1, -0.2], ds_overlap=0.4)
    st = run(sc)
    dds = 0.6 * D0
    assert abs((st.x[1] - st.x[0]) - dds) < 1e-15
    assert np.allclose(st.z, 0.0)
    # momentum of the pair is kept (equal masses)
    assert abs((st.u[0] + st.u[1]) - (0.1 - 0.2)) < 1e-12
    # each particle moved half the deficit, symmetric about the midpoint
    assert abs(0.5 * (st.x[0] + st.x[1]) - 0.5 * r0) < 1e-15


def test_ds_diagonal_pair_and_translation_invariance():
    e = np.array([0.6, 0.8])
    r0 = 0.25 * D0
    base = np.array([0.013, 0.021])
    sc = make([base[0], base[0] + r0 * e[0]], [base[1], base[1] + r0 * e[1]], ds_overlap=0.4)
    st = run(sc)
    sep = np.array([st.x[1] - st.x[0], st.z[1] - st.z[0]])
    assert abs(np.linalg.norm(sep) - 0.6 * D0) < 1e-15
    assert abs(sep[0] * e[1] - sep[1] * e[0]) < 1e-15     # still along e
    sc2 = make([0.5 + base[0], 0.5 + base[0] + r0 * e[0]], [base[1], base[1] + r0 * e[1]],
               ds_overlap=0.4)
    st2 = run(sc2)
    assert np.allclose(st2.x - 0.5, st.x, atol=1e-15) and np.allclose(st2.z, st.z, atol=1e-15)


def test_ds_against_wall_moves_fluid_by_whole_deficit():
    r0 = 0.2 * D0
    sc = make([0.0, 0.0], [0.0, r0], types=[S.WALL, S.FLUID], ds_overlap=0.4)
    st = run(sc)
    assert st.z[0] == 0.0 and st.x[0] == 0.0
    assert abs(st.z[1] - 0.6 * D0) < 1e-15
    assert abs(st.w[1] - (0.6 * D0 - r0) / DT) < 1e-9


def test_ds_acts_in_projected_space():
    """E map with alpha = 2: a physical vertical gap of 0.2 d0 is 0.4 d0 in
    projected space; the pair is pushed to 0.6 d0 projected = 0.3 d0 physical."""
    sc = make([0.0, 0.0], [0.0, 0.2 * D0], ds_overlap=0.4, aspect=2.0)
    st = run(sc)
    assert abs((st.z[1] - st.z[0]) - 0.3 * D0) < 1e-15
    # and a physical gap of 0.35 d0 (0.7 d0 projected) is left alone
    sc = make([0.0, 0.0], [0.0, 0.35 * D0], ds_overlap=0.4, aspect=2.0)
    st = run(sc)
    assert np.array_equal(st.z, sc.z) and np.array_equal(st.w, sc.w)


def lattice(nx, nz, jitter=0.0, seed=0):
    rng = np.random.default_rng(seed)
    X, Z = np.meshgrid(np.arange(nx) * D0, np.arange(nz) * D0, indexing="ij")
    x, z = X.ravel().copy(), Z.ravel().copy()
    if jitter:
        x += rng.uniform(-jitter, jitter, x.size) * D0
        z += rng.uniform(-jitter, jitter, x.size) * D0
    return x, z


def test_shift_zero_on_symmetric_lattice_and_at_rest():
    x, z = lattice(11, 11)
    n = x.size
    c = (n - 1) // 2   # centre of the lattice: every neighbour has its mirror image
    u = np.full(n, 0.3)
    st = run(make(x, z, u=u, ops_shift=0.2))
    assert abs(st.x[c] - x[c]) < 1e-18 and abs(st.z[c] - z[c]) < 1e-18
    xj, zj = lattice(11, 11, jitter=0.1, seed=3)
    st = run(make(xj, zj, ops_shift=0.2))            # at rest: D = 0
    assert np.array_equal(st.x, xj) and np.array_equal(st.z, zj)


def test_shift_restores_displaced_particle():
    x, z = lattice(11, 11)
    c = (x.size - 1) // 2
    site = np.array([x[c], z[c]])
    for d in ([0.2, 0.0], [0.0, -0.15], [0.1, 0.12]):
        xd, zd = x.copy(), z.copy()
        xd[c] += d[0] * D0
        zd[c] += d[1] * D0
        st = run(make(xd, zd, u=np.full(x.size, 0.5), ops_shift=0.2))
        moved = np.array([st.x[c] - xd[c], st.z[c] - zd[c]])
        back = site - np.array([xd[c], zd[c]])
        assert moved @ back > 0.0
        assert np.linalg.norm(moved) < np.linalg.norm(back)


def test_shift_of_free_surface_particles_is_tangential():
    """On a regular lattice with a flat top, the top row's concentration
    gradient is normal to the surface: unflagged, those particles are shifted
    out of the fluid (towards lower concentration, the reason the method
    treats the surface apart); flagged as free surface, they stay (only the tangential
    part is kept, and there is none).  Disorder along the top row makes them
    move along it."""
    x, z = lattice(15, 6)
    top = np.isclose(z, z.max())
    inner = top & (np.abs(x - x.mean()) < 3 * D0)
    sc = make(x, z, u=np.full(x.size, 0.4), ops_shift=0.2)
    st = run(sc, fs=np.zeros(x.size, np.int32))
    assert (st.z[inner] - z[inner]).min() > 1e-9           # pushed out of the fluid
    assert np.abs(st.x[inner] - x[inner]).max() < 1e-18
    st = run(sc, fs=top.astype(np.int32))
    assert np.abs(st.z[inner] - z[inner]).max() < 1e-18
    assert np.abs(st.x[inner] - x[inner]).max() < 1e-18
    rng = np.random.default_rng(1)
    xd = x + np.where(top, rng.uniform(-0.1, 0.1, x.size) * D0, 0.0)
    st = run(make(xd, z, u=np.full(x.size, 0.4), ops_shift=0.2), fs=top.astype(np.int32))
    dx, dz = st.x[inner] - xd[inner], st.z[inner] - z[inner]
    assert np.abs(dx).max() > 0.0
    assert np.abs(dz).max() < 0.2 * np.abs(dx).max()      # mostly along the surface


def test_xsph_uniform_field_and_interior_untouched():
    x, z = lattice(9, 9, jitter=0.1, seed=5)
    n = x.size
    fs = (np.arange(n) % 3 == 0).astype(np.int32)
    st = run(make(x, z, u=np.full(n, 0.7), w=np.full(n, -0.2), xsph_eps=5e-3), fs=fs)
    assert np.allclose(st.u, 0.7, rtol=0, atol=1e-15) and np.allclose(st.w, -0.2, rtol=0, atol=1e-15)
    rng = np.random.default_rng(2)
    u, w = rng.normal(size=n), rng.normal(size=n)
    st = run(make(x, z, u=u, w=w, xsph_eps=5e-3), fs=fs)
    interior = fs == 0
    assert np.array_equal(st.u[interior], u[interior]) and np.array_equal(st.w[interior], w[interior])
    assert np.abs(st.u[~interior] - u[~interior]).max() > 0.0
    assert np.array_equal(st.x, x) and np.array_equal(st.z, z)


def test_xsph_pulls_pair_velocities_together():
    sc = make([0.0, 0.9 * D0], [0.0, 0.0], u=[1.0, -1.0], w=[0.0, 0.5], xsph_eps=5e-3)
    st = run(sc, fs=np.array([1, 1], np.int32))
    before = np.hypot(sc.u[0] - sc.u[1], sc.w[0] - sc.w[1])
    after = np.hypot(st.u[0] - st.u[1], st.w[0] - st.w[1])
    assert after < before
    assert abs((st.u[0] + st.u[1]) - 0.0) < 1e-15      # symmetric pair: mean kept
