"""Derivatives of the corrected gradient (sph2_gradient_backward_positions) and
of the SPH(2) second derivatives (sph2_d2_backward_positions) with respect to
the projected particle positions: against central differences of
the oracle's outputs (Eqs. gra_1st, sec_SPH2) in each projected coordinate of fluid and
wall particles, with the neighbour sets unchanged by the step, in 2-D (E map,
aspect 1) and 3-D (E map, aspect 2: a projected step dz^ is a physical step
dz^ / 2); and, at the 2-D wave's size, the invariance of the loss under a
rigid translation (the gradient sums to zero over the particles)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vct():
    from paper_2607_28872_b300 import vct as V
    V.load_library()
    return V


CASES = [
    ("e2d", lambda: S.small_tank(dim=2, kind="E", L=0.16, H=0.06, d0=0.01, seed=3, aspect=1.0,
                                 bathy=S.Bathymetry(), jitter=0.1), 1.0),
    ("e3d", lambda: S.small_tank(dim=3, kind="E", L=0.07, W=0.05, H=0.05, d0=0.01, seed=4,
                                 aspect=2.0, bathy=S.Bathymetry(), jitter=0.1), 2.0),
]


@pytest.mark.parametrize("name,make,aspect", CASES, ids=[c[0] for c in CASES])
def test_position_gradient_matches_oracle_differences(vct, name, make, aspect):
    import torch
    sc = make()
    d, n = sc.dim, sc.n
    rng = np.random.default_rng(21)
    phi = rng.normal(size=(2, n))
    gbar = rng.normal(size=(2, d, n))
    solver = vct.Solver(sc)
    st = vct.DeviceState(sc)
    xb = solver.sph2_gradient_backward_positions(st, torch.tensor(phi), torch.tensor(gbar))
    xb = xb.cpu().numpy()
    assert np.all(xb[:, sc.type == S.VIRTUAL] == 0.0)
    l, re, re2 = O.radii(sc)
    xh0, _ = O.projected(sc)
    row0, col0 = O.neighbours(d, xh0, re, re2, mode=0)
    eps = 1e-7 * sc.params["d0"]
    names = ("x", "y", "z") if d == 3 else ("x", "z")
    picks = list(np.flatnonzero(sc.type == S.FLUID)[::17][:6]) + \
        list(np.flatnonzero(sc.type == S.WALL)[::11][:3])
    scale = np.abs(xb).max()
    for p in picks:
        for K, nm in enumerate(names):
            step = eps / aspect if nm == "z" else eps
            vals = []
            for sgn in (1.0, -1.0):
                s2 = sc.copy()
                getattr(s2, nm)[p] += sgn * step
                xh, _ = O.projected(s2)
                row, col = O.neighbours(d, xh, re, re2, mode=0)
                assert np.array_equal(row, row0) and np.array_equal(col, col0)
                g, _, _ = O.sph2_derivatives(s2, phi)
                vals.append(np.sum(gbar * g))
            fd = (vals[0] - vals[1]) / (2 * eps)
            assert abs(fd - xb[K, p]) <= 1e-6 * scale, (p, nm, fd, xb[K, p])


def test_position_gradient_translation_invariance(vct):
    import torch
    sc = S.solitary_sigma(precision=0)
    rng = np.random.default_rng(22)
    phi = rng.normal(size=(1, sc.n))
    gbar = rng.normal(size=(1, sc.dim, sc.n))
    solver = vct.Solver(sc)
    xb = solver.sph2_gradient_backward_positions(vct.DeviceState(sc), torch.tensor(phi),
                                                 torch.tensor(gbar)).cpu().numpy()
    assert np.abs(xb).max() > 0.0
    for K in range(sc.dim):
        assert abs(xb[K].sum()) <= 1e-10 * np.abs(xb[K]).sum()


@pytest.mark.parametrize("name,make,aspect", CASES, ids=[c[0] for c in CASES])
def test_second_derivative_position_gradient_matches_oracle_differences(vct, name, make, aspect):
    import torch
    sc = make()
    d, n = sc.dim, sc.n
    m = 3 if d == 2 else 6
    rng = np.random.default_rng(23)
    phi = rng.normal(size=n)
    dbar = rng.normal(size=(m, n))
    solver = vct.Solver(sc)
    xb = solver.sph2_d2_backward_positions(vct.DeviceState(sc), torch.tensor(phi),
                                           torch.tensor(dbar)).cpu().numpy()
    assert np.all(xb[:, sc.type == S.VIRTUAL] == 0.0)
    l, re, re2 = O.radii(sc)
    xh0, _ = O.projected(sc)
    row0, col0 = O.neighbours(d, xh0, re, re2, mode=0)
    eps = 1e-7 * sc.params["d0"]
    names = ("x", "y", "z") if d == 3 else ("x", "z")
    picks = list(np.flatnonzero(sc.type == S.FLUID)[::19][:5]) + \
        list(np.flatnonzero(sc.type == S.WALL)[::13][:3])
    scale = np.abs(xb).max()
    for p in picks:
        for K, nm in enumerate(names):
            step = eps / aspect if nm == "z" else eps
            vals = []
            for sgn in (1.0, -1.0):
                s2 = sc.copy()
                getattr(s2, nm)[p] += sgn * step
                xh, _ = O.projected(s2)
                row, col = O.neighbours(d, xh, re, re2, mode=0)
                assert np.array_equal(row, row0) and np.array_equal(col, col0)
                _, d2, _ = O.sph2_derivatives(s2, phi[None, :])
                vals.append(np.sum(dbar * d2[0]))
            fd = (vals[0] - vals[1]) / (2 * eps)
            assert abs(fd - xb[K, p]) <= 1e-6 * scale, (p, nm, fd, xb[K, p])
    for K in range(d):   # rigid translation leaves the outputs unchanged
        assert abs(xb[K].sum()) <= 1e-10 * np.abs(xb[K]).sum()


def test_second_derivative_position_gradient_needs_scratch(vct):
    import torch
    sc = CASES[0][1]()
    solver = vct.Solver(sc, max_neighbours=24)
    with pytest.raises(vct.VCTError) as e:
        solver.sph2_d2_backward_positions(vct.DeviceState(sc), torch.zeros(sc.n),
                                          torch.zeros((3, sc.n)))
    assert e.value.status == vct.VCT_ERR_CAPACITY


@pytest.mark.parametrize("name,make,aspect", CASES, ids=[c[0] for c in CASES])
def test_pressure_operator_position_gradient_matches_oracle_differences(vct, name, make, aspect):
    """pbar . (A x) with the oracle's operator (its probe of A x_test), x zero
    off the unknown rows, free-surface flags and neighbour sets checked
    unchanged by each step (maps with a constant metric: E)."""
    import torch
    sc = make()
    d, n = sc.dim, sc.n
    _, info0 = O.step(sc, probe=True, rtol=1e-13)
    fs0 = info0["fs"]
    unknown = (sc.type == S.FLUID) & (fs0 == 0)
    rng = np.random.default_rng(24)
    x = np.where(unknown, rng.normal(size=n), 0.0)
    pbar = rng.normal(size=n)
    solver = vct.Solver(sc)
    xb = solver.vct_ppe_backward_positions(vct.DeviceState(sc), torch.tensor(x),
                                           torch.tensor(pbar)).cpu().numpy()
    assert np.all(xb[:, sc.type == S.VIRTUAL] == 0.0)
    l, re, re2 = O.radii(sc)
    xh0, _ = O.projected(sc)
    row0, col0 = O.neighbours(d, xh0, re, re2, mode=0)
    eps = 1e-7 * sc.params["d0"]
    names = ("x", "y", "z") if d == 3 else ("x", "z")
    picks = list(np.flatnonzero(unknown)[::19][:5]) + list(np.flatnonzero(sc.type == S.WALL)[::13][:3])
    scale = np.abs(xb).max()
    for p in picks:
        for K, nm in enumerate(names):
            step = eps / aspect if nm == "z" else eps
            vals = []
            for sgn in (1.0, -1.0):
                s2 = sc.copy()
                getattr(s2, nm)[p] += sgn * step
                xh, _ = O.projected(s2)
                row, col = O.neighbours(d, xh, re, re2, mode=0)
                assert np.array_equal(row, row0) and np.array_equal(col, col0)
                _, info = O.step(s2, probe=True, x_test=x, rtol=1e-13)
                assert np.array_equal(info["fs"], fs0)
                vals.append(np.sum(pbar[unknown] * info["ppe_Ax"][unknown]))
            fd = (vals[0] - vals[1]) / (2 * eps)
            assert abs(fd - xb[K, p]) <= 1e-6 * scale, (p, nm, fd, xb[K, p])


@pytest.mark.parametrize("name,make,aspect", CASES, ids=[c[0] for c in CASES])
def test_density_position_gradient_matches_oracle_differences(vct, name, make, aspect):
    """rhobar . rho^ with the oracle's density estimate (its probe), neighbour
    sets checked unchanged by each step."""
    import torch
    sc = make()
    d, n = sc.dim, sc.n
    rng = np.random.default_rng(25)
    rbar = rng.normal(size=n)
    solver = vct.Solver(sc)
    xb = solver.vct_rho_backward_positions(vct.DeviceState(sc), torch.tensor(rbar)).cpu().numpy()
    fluid = sc.type == S.FLUID
    l, re, re2 = O.radii(sc)
    xh0, _ = O.projected(sc)
    row0, col0 = O.neighbours(d, xh0, re, re2, mode=0)
    eps = 1e-7 * sc.params["d0"]
    names = ("x", "y", "z") if d == 3 else ("x", "z")
    picks = list(np.flatnonzero(fluid)[::19][:4]) + list(np.flatnonzero(sc.type == S.WALL)[::13][:2]) + \
        list(np.flatnonzero(sc.type == S.VIRTUAL)[::13][:2])
    scale = np.abs(xb).max()
    for p in picks:
        for K, nm in enumerate(names):
            step = eps / aspect if nm == "z" else eps
            vals = []
            for sgn in (1.0, -1.0):
                s2 = sc.copy()
                getattr(s2, nm)[p] += sgn * step
                xh, _ = O.projected(s2)
                row, col = O.neighbours(d, xh, re, re2, mode=0)
                assert np.array_equal(row, row0) and np.array_equal(col, col0)
                _, info = O.step(s2, probe=True, rtol=1e-13)
                vals.append(np.sum(rbar[fluid] * info["rho_hat"][fluid]))
            fd = (vals[0] - vals[1]) / (2 * eps)
            assert abs(fd - xb[K, p]) <= 1e-6 * scale, (p, nm, fd, xb[K, p])
    for K in range(d):
        assert abs(xb[K].sum()) <= 1e-10 * np.abs(xb[K]).sum()
