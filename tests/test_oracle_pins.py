"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant, a finite-difference derivative, brute force, or a
library solve.  A plausible slip in the oracle (dropped term, wrong sign,
transposed operand, wrong kernel constant) fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S


# --------------------------------------------------------------------------
# Kernel (Sec. 3.1): unity condition and smoothness of the cubic spline.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_unity_and_derivative(dim):
    l = 0.37
    r = np.linspace(0.0, 2.2 * l, 400001)
    w, dw = O.kernel(dim, l, r)
    shell = 2 * math.pi * r if dim == 2 else 4 * math.pi * r * r
    integral = np.trapezoid(w * shell, r)
    assert abs(integral - 1.0) < 1e-9
    # w' is the derivative of w (central differences)
    fd = np.gradient(w, r)
    assert np.max(np.abs(fd[5:-5] - dw[5:-5])) < 1e-4 * np.max(np.abs(dw))
    # C1 at r = l and support ends at 2l with w = w' = 0
    for rr in (l, 2 * l):
        a, da = O.kernel(dim, l, np.array([rr * (1 - 1e-12), rr * (1 + 1e-12)]))
        assert abs(a[0] - a[1]) < 1e-9 * abs(w).max()
        assert abs(da[0] - da[1]) < 1e-9 * abs(dw).max()
    assert w[r >= 2 * l].max() == 0.0


# --------------------------------------------------------------------------
# Map (Sec. 2.2): alpha, beta derivatives against finite differences; Jacobian
# column (Eq. jacobi) against finite differences of the forward map.
# --------------------------------------------------------------------------
def _map_scenarios():
    bump = S.Bathymetry(h0=0.01, slope_x=0.05, slope_y=-0.02, cos_amp=0.01, cos_len=0.7,
                        amp=[0.05, -0.03], cx=[0.3, 0.6], cy=[0.1, 0.25], width=[0.1, 0.15])
    out = []
    for kind, aspect in (("E", 2.5), ("BF", 1.0), ("BFE", 2.0), ("SIGMA", 1.0)):
        sc = S.small_tank(dim=3, kind=kind, L=0.2, W=0.1, H=0.1, d0=0.02, aspect=aspect,
                          bathy=bump, alpha_min=0.5, alpha_max=4.0, H_hat=0.12)
        out.append(sc)
    return out


@pytest.mark.parametrize("sc", _map_scenarios(), ids=lambda s: s.map_kind)
def test_map_derivatives_fd(sc):
    rng = np.random.default_rng(3)
    x = rng.uniform(0.05, 0.95, 64)
    y = rng.uniform(0.0, 0.3, 64)
    h = 1e-4
    ab = O.map_coeffs(sc, x, y)
    for comp, (i_f, i_fx, i_fy, i_fxx, i_fyy) in {"alpha": (0, 1, 2, 3, 4), "beta": (5, 6, 7, 8, 9)}.items():
        fpx = O.map_coeffs(sc, x + h, y)[:, i_f]
        fmx = O.map_coeffs(sc, x - h, y)[:, i_f]
        fpy = O.map_coeffs(sc, x, y + h)[:, i_f]
        fmy = O.map_coeffs(sc, x, y - h)[:, i_f]
        f0 = ab[:, i_f]
        # skip points next to the sigma clamp, where alpha is only C0
        ok = np.ones_like(x, dtype=bool)
        if sc.map_kind == "SIGMA":
            D = sc.params["H"] - sc.bathy.height(x, y)
            a = sc.params["H_hat"] / D
            ok = (np.abs(a - 0.5) > 0.05) & (np.abs(a - 4.0) > 0.05)
        scale = 1.0 + np.abs(f0).max()
        assert np.allclose(((fpx - fmx) / (2 * h))[ok], ab[ok, i_fx], atol=1e-6 * scale), comp
        assert np.allclose(((fpy - fmy) / (2 * h))[ok], ab[ok, i_fy], atol=1e-6 * scale), comp
        assert np.allclose(((fpx - 2 * f0 + fmx) / h ** 2)[ok], ab[ok, i_fxx], atol=1e-3 * scale), comp
        assert np.allclose(((fpy - 2 * f0 + fmy) / h ** 2)[ok], ab[ok, i_fyy], atol=1e-3 * scale), comp


def test_sigma_map_definition_and_clamp():
    sc = _map_scenarios()[3]
    x = np.linspace(0.0, 1.0, 201)
    y = np.full_like(x, 0.1)
    ab = O.map_coeffs(sc, x, y)
    h = sc.bathy.height(x, y)
    a = sc.params["H_hat"] / (sc.params["H"] - h)
    inside = (a >= 0.5) & (a <= 4.0)
    assert np.allclose(ab[inside, 0], a[inside], rtol=1e-14)
    assert np.allclose(ab[:, 5], -h, rtol=1e-14, atol=1e-16)
    assert np.all(ab[~inside, 1:5] == 0.0)          # constant alpha where clamped
    assert np.all((ab[:, 0] >= 0.5) & (ab[:, 0] <= 4.0))


@pytest.mark.parametrize("sc", _map_scenarios(), ids=lambda s: s.map_kind)
def test_jacobian_column_fd(sc):
    rng = np.random.default_rng(4)
    x = rng.uniform(0.05, 0.95, 50)
    y = rng.uniform(0.0, 0.3, 50)
    z = rng.uniform(-0.05, 0.2, 50)
    h = 1e-5
    zh, met = O.map_metric(sc, x, y, z)
    sx = (O.map_metric(sc, x + h, y, z)[0] - O.map_metric(sc, x - h, y, z)[0]) / (2 * h)
    sy = (O.map_metric(sc, x, y + h, z)[0] - O.map_metric(sc, x, y - h, z)[0]) / (2 * h)
    sz = (O.map_metric(sc, x, y, z + h)[0] - O.map_metric(sc, x, y, z - h)[0]) / (2 * h)
    ok = np.ones_like(x, dtype=bool)
    if sc.map_kind == "SIGMA":
        a = sc.params["H_hat"] / (sc.params["H"] - sc.bathy.height(x, y))
        ok = (np.abs(a - 0.5) > 0.05) & (np.abs(a - 4.0) > 0.05)
    assert np.allclose(sx[ok], met[ok, 1], atol=1e-7)
    assert np.allclose(sy[ok], met[ok, 2], atol=1e-7)
    assert np.allclose(sz, met[:, 0], atol=1e-7)      # d z^/dz = alpha = det J
    assert np.allclose(met[:, 5], 2 * met[:, 1]) and np.allclose(met[:, 6], 2 * met[:, 2])


@pytest.mark.parametrize("sc", _map_scenarios(), ids=lambda s: s.map_kind)
def test_c_trans_composite_laplacian(sc):
    """psi quadratic in projected coordinates; the physical Laplacian of
    psi(x, y, alpha (z + beta)) by 4th-order finite differences equals
    c_trans . D^ psi with the exact projected derivatives (Eq. lap_VCT)."""
    A = dict(z=0.7, xx=1.3, yy=-0.4, zz=2.1, xz=0.9, yz=-1.1, xy=0.5, x=0.2, y=-0.3)

    def psi(x, y, z):
        zh, _ = O.map_metric(sc, x, y, z)
        return (A["x"] * x + A["y"] * y + A["z"] * zh + 0.5 * A["xx"] * x * x + 0.5 * A["yy"] * y * y
                + 0.5 * A["zz"] * zh * zh + A["xz"] * x * zh + A["yz"] * y * zh + A["xy"] * x * y)

    rng = np.random.default_rng(5)
    x = rng.uniform(0.05, 0.95, 40)
    y = rng.uniform(0.0, 0.3, 40)
    z = rng.uniform(-0.05, 0.2, 40)
    h = 2e-3

    def d2(axis):
        e = [np.zeros(40)] * 3
        e = [np.full(40, h) if k == axis else np.zeros(40) for k in range(3)]
        f = lambda s: psi(x + s * e[0], y + s * e[1], z + s * e[2])
        return (-f(2) + 16 * f(1) - 30 * f(0) + 16 * f(-1) - f(-2)) / (12 * h * h)

    lap_fd = d2(0) + d2(1) + d2(2)
    zh, met = O.map_metric(sc, x, y, z)
    Dz = A["z"] + A["zz"] * zh + A["xz"] * x + A["yz"] * y
    lap = met[:, 3] * Dz + A["xx"] + A["yy"] + met[:, 4] * A["zz"] + met[:, 5] * A["xz"] + met[:, 6] * A["yz"]
    ok = np.ones_like(x, dtype=bool)
    if sc.map_kind == "SIGMA":
        a = sc.params["H_hat"] / (sc.params["H"] - sc.bathy.height(x, y))
        ok = (np.abs(a - 0.5) > 0.1) & (np.abs(a - 4.0) > 0.1)
    assert np.allclose(lap_fd[ok], lap[ok], rtol=2e-5, atol=2e-5 * np.abs(lap).max())


# --------------------------------------------------------------------------
# Neighbour sets (Eq. SPH_neighbor_set).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,count", [(2, 20), (3, 56)])
def test_neighbour_lattice_count_and_symmetry(dim, count):
    """On a regular lattice with r_e = 2.4 d0 the neighbours are the lattice
    points with |n|^2 in {1,2,4,5}: 4+4+4+8 = 20 in 2-D, 6+12+8+6+24 = 56 in 3-D."""
    sc = S.small_tank(dim=dim, kind="BF", L=0.2, W=0.12, H=0.12, d0=0.01, jitter=0.0,
                      bathy=S.Bathymetry())
    xh, _ = O.projected(sc)
    l, re, re2 = O.radii(sc)
    row, col = O.neighbours(dim, xh, re, re2, mode=0)
    cnt = np.diff(row)
    lo = xh.min(axis=1) + 3 * re
    hi = xh.max(axis=1) - 3 * re
    inner = np.all((xh.T > lo) & (xh.T < hi), axis=1)
    assert inner.sum() > 10
    assert np.all(cnt[inner] == count)
    # symmetric relation
    pairs = set(zip(np.repeat(np.arange(sc.n), cnt).tolist(), col.tolist()))
    assert all((j, i) in pairs for i, j in pairs)


@pytest.mark.parametrize("dim", [2, 3])
def test_neighbour_grid_equals_brute(dim):
    sc = S.small_tank(dim=dim, kind="SIGMA", L=0.25, W=0.1, H=0.08, d0=0.01, seed=7)
    xh, _ = O.projected(sc)
    l, re, re2 = O.radii(sc)
    r0, c0 = O.neighbours(dim, xh, re, re2, mode=0)
    r1, c1 = O.neighbours(dim, xh, re, re2, mode=1)
    assert np.array_equal(r0, r1) and np.array_equal(c0, c1)
    # brute-force definition written directly with numpy
    X = xh.T
    i = 17
    d2 = ((X - X[i]) ** 2).sum(axis=1)
    ref = np.nonzero(d2 < re2)[0]
    ref = ref[ref != i]
    assert np.array_equal(np.sort(ref), c0[r0[i]:r0[i + 1]])


# --------------------------------------------------------------------------
# SPH(2) (Eq. sec_SPH2): exact for quadratics on disordered particles,
# corrected gradient exact for linear fields (Eq. gra_1st).
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,kind", [(2, "BF"), (2, "SIGMA"), (3, "BFE"), (3, "SIGMA")])
def test_sph2_quadratic_exact(dim, kind):
    sc = S.small_tank(dim=dim, kind=kind, L=0.2, W=0.08, H=0.08, d0=0.01, seed=11, jitter=0.2,
                      aspect=2.0)
    f = sc.type == S.FLUID
    xh, met = O.projected(sc)
    rng = np.random.default_rng(1)
    m = 3 if dim == 2 else 6
    H = rng.normal(size=(dim, dim))
    H = H + H.T
    a = rng.normal(size=dim)
    X = xh
    phi = 0.4 + a @ X + 0.5 * np.einsum("kn,kl,ln->n", X, H, X)
    lin = 0.4 + a @ X
    g, d2, lap = O.sph2_derivatives(sc, np.stack([phi, lin]))
    if dim == 2:
        exact = [H[0, 0], H[1, 1], H[0, 1]]
    else:
        exact = [H[0, 0], H[1, 1], H[2, 2], H[0, 1], H[1, 2], H[2, 0]]
    scale = np.abs(H).max()
    for k in range(m):
        assert np.abs(d2[0, k, f] - exact[k]).max() < 1e-8 * scale
        assert np.abs(d2[1, k, f]).max() < 1e-8 * scale
    for K in range(dim):
        assert np.abs(g[1, K, f] - a[K]).max() < 1e-11 * np.abs(a).max()
    # composite: c_trans . D^ phi with the exact projected derivatives
    vert = dim - 1
    dz = a[vert] + H[vert] @ X
    if dim == 2:
        ref = met[:, 3] * dz + H[0, 0] + met[:, 4] * H[1, 1] + met[:, 5] * H[0, 1]
    else:
        ref = (met[:, 3] * dz + H[0, 0] + H[1, 1] + met[:, 4] * H[2, 2] + met[:, 5] * H[0, 2]
               + met[:, 6] * H[1, 2])
    # the gradient entering c0 is first-order, so compare where c0 == 0 exactly
    # (BF/BFE linear pieces) or allow the first-order gradient error otherwise
    err = np.abs(lap[0, f] - ref[f] + met[f, 3] * (dz[f] - g[0, vert, f]))
    assert err.max() < 1e-7 * (np.abs(ref).max() + 1)


def test_sph2_second_order_convergence():
    """Laplacian and cross derivative of a smooth field on regular lattices:
    error ratio ~4 per halving of d0 (second-order consistency, Sec. 3.1)."""
    errs = []
    k = 2 * math.pi / 0.4
    for d0 in (0.02, 0.01, 0.005):
        sc = S.small_tank(dim=2, kind="BF", L=0.4, H=0.4, d0=d0, jitter=0.0,
                          bathy=S.Bathymetry())
        f = sc.type == S.FLUID
        xh, _ = O.projected(sc)
        X, Z = xh
        phi = np.sin(k * X) * np.cos(0.7 * k * Z)
        g, d2, lap = O.sph2_derivatives(sc, phi[None])
        core = f & (X > 0.12) & (X < 0.28) & (Z > 0.12) & (Z < 0.28)
        exx = -k * k * phi
        exz = -k * 0.7 * k * np.cos(k * X) * np.sin(0.7 * k * Z)
        errs.append((np.abs(d2[0, 0, core] - exx[core]).max(), np.abs(d2[0, 2, core] - exz[core]).max()))
    for a, b in zip(errs[:-1], errs[1:]):
        assert math.log2(a[0] / b[0]) > 1.8
        assert math.log2(a[1] / b[1]) > 1.8


# --------------------------------------------------------------------------
# Volume smoothing (Sec. 3.6): sum_i J_i / Jbar_i is conserved.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
def test_volume_smoothing_conserves(mode):
    sc = S.small_tank(dim=2, kind="SIGMA", L=0.3, H=0.1, d0=0.01, seed=2)
    st = O.OracleState(sc)
    f = sc.type == S.FLUID
    rng = np.random.default_rng(9)
    _, met = O.projected(sc)
    J = met[:, 0]
    st.jbar[:] = J * rng.uniform(0.8, 1.25, sc.n)   # uneven volumes to exchange
    before = np.sum(J[f] / st.jbar[f])
    O.volume_smoothing(sc, st, mode)
    after = np.sum(J[f] / st.jbar[f])
    assert abs(after - before) < 1e-12 * before
    assert np.std(J[f] / st.jbar[f]) < np.std(J[f] / (J[f] * rng.uniform(0.8, 1.25, f.sum()))) * 2


# --------------------------------------------------------------------------
# Pressure equation: operator on quadratics, BiCGSTAB vs a dense solve.
# --------------------------------------------------------------------------
def test_ppe_operator_on_quadratic():
    sc = S.small_tank(dim=2, kind="SIGMA", L=0.3, H=0.12, d0=0.01, seed=3, jitter=0.1)
    f = sc.type == S.FLUID
    xh, met = O.projected(sc)
    X, Z = xh
    xt = 1.0 + 0.3 * X - 0.2 * Z + 0.5 * 2.0 * X * X + 0.5 * 1.5 * Z * Z - 0.7 * X * Z
    _, info = O.step(sc, probe=True, x_test=xt)
    fs = info["fs"] == 1
    l, re, re2 = O.radii(sc)
    row, col = O.neighbours(2, xh, re, re2)
    interior = np.zeros(sc.n, dtype=bool)
    for i in np.nonzero(f & ~fs)[0]:
        nb = col[row[i]:row[i + 1]]
        interior[i] = np.all(f[nb] & ~fs[nb])
    assert interior.sum() > 50
    dz = -0.2 + 1.5 * Z - 0.7 * X
    ref = met[:, 3] * dz + 2.0 + met[:, 4] * 1.5 + met[:, 5] * (-0.7)
    # c0 multiplies the first-order gradient, whose error is O(d0) for a quadratic
    g, _, _ = O.sph2_derivatives(sc, xt[None])
    ref_discrete = ref - met[:, 3] * (dz - g[0, 1])
    assert np.allclose(info["ppe_Ax"][interior], ref_discrete[interior], rtol=1e-8, atol=1e-8)


def test_ppe_bicgstab_matches_dense_solve():
    sc = S.small_tank(dim=2, kind="BF", L=0.12, H=0.08, d0=0.01, seed=5, jitter=0.1,
                      bathy=S.Bathymetry(h0=-0.01, slope_x=0.1))
    n = sc.n
    st, info = O.step(sc, probe=True)
    unk = np.nonzero((sc.type == S.FLUID) & (info["fs"] == 0))[0]
    A = np.zeros((unk.size, unk.size))
    for c, j in enumerate(unk):
        e = np.zeros(n)
        e[j] = 1.0
        _, inf2 = O.step(sc, probe=True, x_test=e)
        A[:, c] = inf2["ppe_Ax"][unk]
    b = info["ppe_b"][unk]
    p_dense = np.linalg.solve(A, b)
    assert np.allclose(st.p[unk], p_dense, rtol=1e-9, atol=1e-9 * np.abs(p_dense).max())
    assert info["resid"] < 1e-12


# --------------------------------------------------------------------------
# Free surface (reading of Sec. 3.5) and still water (P2).
# --------------------------------------------------------------------------
def test_free_surface_is_top_layer_of_regular_block():
    sc = S.small_tank(dim=2, kind="E", L=0.3, H=0.1, d0=0.01, jitter=0.0, aspect=1.5,
                      bathy=S.Bathymetry())
    _, info = O.step(sc, probe=True)
    f = sc.type == S.FLUID
    ztop = np.max(sc.z[f])
    top = f & (np.abs(sc.z - ztop) < 1e-9)
    assert np.array_equal(info["fs"][f] == 1, top[f])


@pytest.mark.parametrize("kind,aspect", [("BF", 1.0), ("E", 2.5), ("BFE", 2.0)])
def test_still_water_exactly_at_rest(kind, aspect):
    """Linear bottom, regular projected lattice, no stabilisation source:
    hydrostatic p is linear in projected coordinates, so J grad^ p + rho g = 0
    holds exactly in the corrected gradient and the PPE right side vanishes;
    the water stays at rest to roundoff."""
    sc = S.small_tank(dim=2, kind=kind, L=0.3, H=0.1, d0=0.01, jitter=0.0, aspect=aspect,
                      bathy=S.Bathymetry(h0=-0.015, slope_x=0.1) if kind != "E" else S.Bathymetry(),
                      gamma_over_dt=0.0)
    f = sc.type == S.FLUID
    st, info = O.step(sc, nsteps=20)
    assert info["rc"] == 0
    vmax = np.sqrt(st.u ** 2 + st.w ** 2)[f].max()
    assert vmax < 1e-10
    assert np.allclose(st.p[f], sc.p[f], atol=1e-8 * sc.p.max())


def test_still_water_jittered_bounded():
    """The jittered still-water tank as specified (jitter 0.1 d0, gamma = 100 dt): the density
    relaxation of the stabilised PPE moves particles, but 20 steps stay
    bounded and the pressure stays near hydrostatic."""
    sc = S.still_water_bf()
    f = sc.type == S.FLUID
    st, info = O.step(sc, nsteps=20, probe=True)
    assert info["rc"] == 0
    vmax = np.sqrt(st.u ** 2 + st.w ** 2)[f].max()
    assert vmax < 0.15
    keep = f & (info["fs"] == 0)
    hyd = sc.params["rho"] * sc.params["g"] * (sc.params["H"] - st.z)
    rel = np.linalg.norm((st.p - hyd)[keep]) / np.linalg.norm(hyd[keep])
    assert rel < 0.1
