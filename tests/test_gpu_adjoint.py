"""Adjoint of the SPH(2) derivative operator (sph2_derivatives_backward).

Checked three ways: the dot-product identity <J phi, y> = <phi, J^T y> to
roundoff; against the oracle's Jacobian, assembled column by column from the
oracle's forward on a tiny tank (an oracle gradient, no CUDA input); and
through torch.autograd against central differences of the GPU forward.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


def _tiny(kind="SIGMA", dim=2, precision=0):
    if dim == 2:
        return S.small_tank(dim=2, kind=kind, L=0.12, H=0.06, d0=0.01, seed=3, with_wave=True,
                            precision=precision)
    return S.small_tank(dim=3, kind=kind, L=0.06, W=0.05, H=0.04, d0=0.01, seed=4,
                        precision=precision)


@pytest.mark.parametrize("dim,kind", [(2, "SIGMA"), (2, "BF"), (3, "BFE")])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "mixed"])
def test_dot_product_identity(dim, kind, precision, tol):
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = _tiny(kind, dim, precision)
    s = V.Solver(sc)
    st = V.DeviceState(sc)
    rng = np.random.default_rng(0)
    n, m = sc.n, (3 if dim == 2 else 6)
    phi = torch.tensor(rng.normal(size=(2, n)), device="cuda")
    gy = torch.tensor(rng.normal(size=(2, dim, n)), device="cuda")
    dy = torch.tensor(rng.normal(size=(2, m, n)), device="cuda")
    ly = torch.tensor(rng.normal(size=(2, n)), device="cuda")
    g, d2, lap = s.sph2_derivatives(st, phi)
    lhs = float((g * gy).sum() + (d2 * dy).sum() + (lap * ly).sum())
    pb = s.sph2_derivatives_backward(st, gy, dy, ly)
    rhs = float((phi * pb).sum())
    scale = float((g.abs() * gy.abs()).sum() + (d2.abs() * dy.abs()).sum() + (lap.abs() * ly.abs()).sum())
    assert abs(lhs - rhs) <= tol * scale


def test_adjoint_matches_oracle_jacobian():
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = _tiny("SIGMA", 2, 0)
    n = sc.n
    f = sc.type == S.FLUID
    # oracle Jacobian of phi -> lap_phys, column by column
    Jl = np.zeros((n, n))
    Jg = np.zeros((2, n, n))
    for col in range(n):
        e = np.zeros((1, n))
        e[0, col] = 1.0
        g, d2, lap = O.sph2_derivatives(sc, e)
        Jl[:, col] = lap[0]
        Jg[:, :, col] = g[0]
    rng = np.random.default_rng(1)
    _, info = O.step(sc, probe=True)
    ly = rng.normal(size=n) * f * (info["fs"] == 0)    # interior rows: well-conditioned M_i
    gy = rng.normal(size=(2, n)) * f
    ref = Jl.T @ ly + Jg[0].T @ gy[0] + Jg[1].T @ gy[1]
    s = V.Solver(sc)
    pb = s.sph2_derivatives_backward(V.DeviceState(sc), torch.tensor(gy[None], device="cuda"),
                                     None, torch.tensor(ly[None], device="cuda"))
    pb = pb.cpu().numpy()[0]
    assert np.abs(pb - ref).max() <= 1e-11 * np.abs(ref).max()


def test_autograd_matches_central_differences():
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = _tiny("SIGMA", 2, 0)
    s = V.Solver(sc)
    st = V.DeviceState(sc)
    F = V.sph2_function()
    rng = np.random.default_rng(2)
    n = sc.n
    w = torch.tensor(rng.normal(size=(1, n)), device="cuda")
    phi0 = torch.tensor(rng.normal(size=(1, n)), device="cuda")

    def loss(ph):
        g, d2, lap = F.apply(ph, s, st)
        return (w * lap).sum() + 0.5 * (g ** 2).sum()

    phi = phi0.clone().requires_grad_(True)
    L = loss(phi)
    L.backward()
    grad = phi.grad.cpu().numpy()[0]
    h = 1e-6
    for k in rng.choice(np.nonzero(sc.type == S.FLUID)[0], 6, replace=False):
        e = torch.zeros_like(phi0)
        e[0, k] = h
        fd = (float(loss(phi0 + e)) - float(loss(phi0 - e))) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * (abs(fd) + 1.0)


def _theta_vector(b):
    return np.array([b.h0, b.slope_x, b.slope_y, b.cos_amp, b.cos_len] + list(b.amp) + list(b.cx)
                    + list(b.cy) + list(b.width), dtype=np.float64)


def _set_theta(b, th):
    G = len(b.amp)
    b.h0, b.slope_x, b.slope_y, b.cos_amp, b.cos_len = (float(v) for v in th[:5])
    b.amp = list(th[5:5 + G])
    b.cx = list(th[5 + G:5 + 2 * G])
    b.cy = list(th[5 + 2 * G:5 + 3 * G])
    b.width = list(th[5 + 3 * G:5 + 4 * G])


@pytest.mark.parametrize("kind,dim", [("SIGMA", 2), ("BF", 2), ("BFE", 3), ("SIGMA", 3)])
def test_map_backward_matches_oracle_differences(kind, dim):
    """theta_bar from the GPU against central differences of the oracle's metric
    (z^, J, s_x, s_y, c0, c3) for every bathymetry parameter."""
    import copy
    import torch
    from paper_2607_28872_b300 import vct as V
    bathy = S.Bathymetry(h0=0.01, slope_x=0.03, slope_y=-0.02, cos_amp=0.004, cos_len=0.17,
                         amp=[0.02, -0.015], cx=[0.05, 0.09], cy=[0.02, 0.03], width=[0.03, 0.04])
    sc = S.small_tank(dim=dim, kind=kind, L=0.12, W=0.05, H=0.06, d0=0.01, seed=6, bathy=bathy,
                      aspect=2.0, alpha_min=0.5, alpha_max=4.0)
    rng = np.random.default_rng(7)
    n = sc.n
    bars = [rng.normal(size=n) for _ in range(6)]
    s = V.Solver(sc)
    got = s.vct_map_backward(V.DeviceState(sc), *[torch.tensor(b, device="cuda") for b in bars])
    th0 = _theta_vector(sc.bathy)

    def objective(th):
        sc2 = copy.deepcopy(sc)
        _set_theta(sc2.bathy, th)
        zh, met = O.map_metric(sc2, sc.x, sc.y, sc.z)
        q = [zh, met[:, 0], met[:, 1], met[:, 2], met[:, 3], met[:, 4]]
        return sum(float(np.dot(bars[k], q[k])) for k in range(6))

    for k in range(th0.size):
        h = 1e-6 * max(1.0, abs(th0[k]))
        tp, tm = th0.copy(), th0.copy()
        tp[k] += h
        tm[k] -= h
        fd = (objective(tp) - objective(tm)) / (2 * h)
        assert abs(fd - got[k]) <= 1e-5 * (abs(fd) + abs(got[k]) + 1e-3), (k, fd, got[k])


@pytest.mark.parametrize("kind,dim", [("SIGMA", 2), ("BF", 2), ("BFE", 3), ("SIGMA", 3)])
def test_map_backward_positions_matches_oracle_differences(kind, dim):
    """The metric under moving particles: pos_bar from the GPU against central
    differences of the oracle's per-particle metric (z^, J, s_x, s_y, c0, c3) in
    each physical coordinate of every particle, with the sigma clamp active on
    part of the tank (alpha_max 4 over the deepest bump)."""
    import torch
    from paper_2607_28872_b300 import vct as V
    bathy = S.Bathymetry(h0=0.01, slope_x=0.03, slope_y=-0.02, cos_amp=0.004, cos_len=0.17,
                         amp=[0.02, -0.015], cx=[0.05, 0.09], cy=[0.02, 0.03], width=[0.03, 0.04])
    sc = S.small_tank(dim=dim, kind=kind, L=0.12, W=0.05, H=0.06, d0=0.01, seed=6, bathy=bathy,
                      aspect=2.0, alpha_min=0.5, alpha_max=4.0)
    rng = np.random.default_rng(8)
    n = sc.n
    bars = [rng.normal(size=n) for _ in range(6)]
    s = V.Solver(sc)
    got = s.vct_map_backward_positions(V.DeviceState(sc),
                                       *[torch.tensor(b, device="cuda") for b in bars]).cpu().numpy()
    y0 = sc.y if sc.y is not None else np.zeros(n)

    def objective(x, y, z):
        zh, met = O.map_metric(sc, x, y, z)
        q = [zh, met[:, 0], met[:, 1], met[:, 2], met[:, 3], met[:, 4]]
        return np.array([sum(bars[k][i] * q[k][i] for k in range(6)) for i in range(n)])

    coords = [sc.x, y0, sc.z]
    axes = (0, 2) if dim == 2 else (0, 1, 2)
    for k, a in enumerate(axes):
        h = 1e-6
        cp = [c.copy() for c in coords]
        cm = [c.copy() for c in coords]
        cp[a] = cp[a] + h
        cm[a] = cm[a] - h
        fd = (objective(*cp) - objective(*cm)) / (2 * h)
        scale = np.abs(fd).max() + 1e-3
        err = np.abs(fd - got[k]).max() / scale
        print(f"PARITY map positions {kind} {dim}-D axis {a}: err {err:.2e}")
        assert err < 1e-6, (a, err)
