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
