"""Adjoint of the pressure solve (vct_ppe_adjoint) against the oracle.

For the pressure system A p = b of one step (Sec. 3.3, Eqs. VCT_ppe and PNC)
the adjoint is b_bar = A^-T p_bar.  Checked element by element against the
transpose solve of the oracle's dense matrix on small tanks (2-D sigma with a
wave, 2-D BF on a slope, 3-D BFE), and by the adjoint identity
<p_bar, p> = <b_bar, b> with the oracle's own b and p on a larger tank.
Tolerances: the GPU's transpose solve stops at a relative residual of 1e-12;
cond(A) of these systems is ~1e2 (measured on the oracle's dense matrices), so
FP64 agrees to 1e-9; the mixed form's operator has FP32 coefficients (relative
1e-7 each), so its adjoint agrees to 1e-4, the bound of the mixed pressure.
"""
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


def rel(g, o):
    return np.abs(g - o).max() / np.abs(o).max()


TANKS = [
    ("sigma2d", lambda: S.small_tank(dim=2, kind="SIGMA", L=0.2, H=0.06, d0=0.01, seed=2,
                                     with_wave=True)),
    ("bf2d", lambda: S.small_tank(dim=2, kind="BF", L=0.25, H=0.08, d0=0.01, seed=1,
                                  bathy=S.Bathymetry(h0=-0.02, slope_x=0.1))),
    ("bfe3d", lambda: S.small_tank(dim=3, kind="BFE", L=0.07, W=0.05, H=0.05, d0=0.01, seed=4,
                                   aspect=2.0)),
]


_SYSTEMS = {}


def _oracle_system(name, sc):
    """The oracle's dense system and probe of one tank (once per tank)."""
    if name not in _SYSTEMS:
        rows, A, b, p = O.ppe_system(sc, rtol=1e-13)
        _, info = O.step(sc, probe=True, rtol=1e-13)
        _SYSTEMS[name] = (rows, A, info["fs"])
    return _SYSTEMS[name]


def _gpu_adjoint(vct, sc, precision, p_bar):
    import torch
    sc = sc.copy()
    sc.params["precision"] = precision
    sc.params["krylov_rtol"] = 1e-12
    sc.params["krylov_max_iter"] = 20000
    solver = vct.Solver(sc)
    st = vct.DeviceState(sc)
    out, _ = solver.vct_step_probe(st)
    b_bar, stats = solver.vct_ppe_adjoint(torch.tensor(p_bar, device="cuda"))
    return out["fs"].cpu().numpy(), b_bar.cpu().numpy(), stats


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-4)], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make", TANKS, ids=[t[0] for t in TANKS])
def test_ppe_adjoint_matches_oracle_transpose_solve(vct, name, make, precision, tol):
    sc = make()
    rows, A, fs_orc = _oracle_system(name, sc)
    rng = np.random.default_rng(11)
    p_bar = rng.normal(size=sc.n)          # entries off the unknown rows must be ignored
    expect = O.ppe_adjoint(A, p_bar[rows])
    fs, b_bar, stats = _gpu_adjoint(vct, sc, precision, p_bar)
    assert np.array_equal(fs, fs_orc), "free-surface flags differ"
    assert stats.steps_done == 1 and stats.krylov_iters_total > 0
    assert stats.last_residual <= 1e-12
    off = np.ones(sc.n, bool)
    off[rows] = False
    assert np.all(b_bar[off] == 0.0)
    assert rel(b_bar[rows], expect) < tol


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-4)], ids=["fp64", "mixed"])
def test_ppe_adjoint_identity_larger_tank(vct, precision, tol):
    """<p_bar, A^-1 b> = <A^-T p_bar, b> with the oracle's b and p (no dense
    matrix: a property that holds at any size)."""
    sc = S.small_tank(dim=2, kind="SIGMA", L=1.0, H=0.1, d0=0.01, seed=3, with_wave=True)
    ost, info = O.step(sc, probe=True, rtol=1e-13)
    unknown = (sc.type == S.FLUID) & (info["fs"] == 0)
    rng = np.random.default_rng(12)
    p_bar = rng.normal(size=sc.n)
    fs, b_bar, _ = _gpu_adjoint(vct, sc, precision, p_bar)
    assert np.array_equal(fs, info["fs"])
    lhs = p_bar[unknown] @ ost.p[unknown]
    rhs = b_bar[unknown] @ info["ppe_b"][unknown]
    scale = np.abs(p_bar[unknown]) @ np.abs(ost.p[unknown])
    assert abs(lhs - rhs) < tol * scale


def test_ppe_adjoint_needs_a_held_system(vct):
    import torch
    sc = TANKS[0][1]()
    solver = vct.Solver(sc)
    st = vct.DeviceState(sc)
    z = torch.zeros(sc.n, dtype=torch.float64, device="cuda")
    with pytest.raises(vct.VCTError) as e:
        solver.vct_ppe_adjoint(z)                       # no step yet
    assert e.value.status == vct.VCT_ERR_ARG
    solver.vct_step(st, 1)
    b_bar, stats = solver.vct_ppe_adjoint(z)            # zero gradient: zero adjoint
    assert torch.count_nonzero(b_bar).item() == 0 and stats.krylov_iters_total == 0
    solver.vct_build_neighbours(st)                     # sorts again: the system is gone
    with pytest.raises(vct.VCTError) as e:
        solver.vct_ppe_adjoint(z)
    assert e.value.status == vct.VCT_ERR_ARG


def test_ppe_adjoint_identity_bumpy_channel(vct):
    """The 2-D channel with 16 random bumps (53k fluid particles, FP64 form):
    the multigrid transpose solve converges (no Jacobi retry: tens of
    iterations, not hundreds) and satisfies the identity with the oracle's b and
    p."""
    sc = S.adjoint_sigma(precision=0)
    sc.params["krylov_rtol"] = 1e-12
    ost, info = O.step(sc, probe=True, rtol=1e-13)
    assert info["rc"] == 0
    unknown = (sc.type == S.FLUID) & (info["fs"] == 0)
    rng = np.random.default_rng(13)
    p_bar = rng.normal(size=sc.n)
    fs, b_bar, stats = _gpu_adjoint(vct, sc, 0, p_bar)
    assert np.array_equal(fs, info["fs"])
    assert stats.krylov_iters_total < 100
    lhs = p_bar[unknown] @ ost.p[unknown]
    rhs = b_bar[unknown] @ info["ppe_b"][unknown]
    scale = np.abs(p_bar[unknown]) @ np.abs(ost.p[unknown])
    assert abs(lhs - rhs) < 1e-7 * scale


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_ppe_adjoint_leaves_the_operator_as_it_was(vct, precision):
    """The transposed solve swaps A's coefficient pairs to stand A^T in A's place
    and swaps them back: two calls in a row give the same b_bar bit for bit (had
    the first left A^T in place, the second would solve with A itself)."""
    import torch
    sc = TANKS[0][1]().copy()
    sc.params["precision"] = precision
    sc.params["krylov_rtol"] = 1e-12
    sc.params["krylov_max_iter"] = 20000
    rng = np.random.default_rng(21)
    p_bar = torch.tensor(rng.normal(size=sc.n), device="cuda")
    solver = vct.Solver(sc)
    solver.vct_step_probe(vct.DeviceState(sc))
    b1, _ = solver.vct_ppe_adjoint(p_bar)
    b2, _ = solver.vct_ppe_adjoint(p_bar)
    assert torch.equal(b1, b2)
