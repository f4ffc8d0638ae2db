"""Closed-form pins of the oracle's predictor and pressure right side.

The terms pinned here vanish in still water, so the rest tests cannot see
them: the viscous term nu c_trans . D^v and the variable-viscosity term
[(grad v) + (grad v)^T] grad nu of Eq. (VCT_predictor), the Smagorinsky eddy
viscosity with its wall damping (Sec. 3.4), and the divergence and
stabilisation source of the pressure right side (Eqs. VCT_ppe, VCT_ppe_w).

Each test prescribes a velocity field for which the continuous term has a
closed form that the discrete operators reproduce exactly: linear fields
(first-order corrected gradients are exact on any neighbourhood), and
quadratic fields on particles whose neighbourhoods are point-symmetric on a
regular projected lattice (the odd moments cancel, so the first-order
gradient is exact too, and SPH(2) is exact for quadratics).  Expected values
come from hand-derived closed forms or from 4th-order finite differences of
the physical field, never from the oracle's own expressions.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S


def _csr(sc):
    xh, met = O.projected(sc)
    _, re, re2 = O.radii(sc)
    row, col = O.neighbours(sc.dim, xh, re, re2)
    return xh, met, row, col


def _full_fluid(sc, row, col, count):
    """Fluid particles whose neighbour set is the complete lattice stencil and
    contains fluid particles only (point-symmetric, no wall values)."""
    f = sc.type == S.FLUID
    out = np.zeros(sc.n, dtype=bool)
    for i in np.flatnonzero(f):
        nb = col[row[i]:row[i + 1]]
        out[i] = nb.size == count and np.all(f[nb])
    return out


def _all_nb(row, col, mask, sel):
    """sel & (every neighbour of i satisfies mask)."""
    out = np.zeros(sel.shape, dtype=bool)
    for i in np.flatnonzero(sel):
        out[i] = np.all(mask[col[row[i]:row[i + 1]]])
    return out


# --------------------------------------------------------------------------
# Viscous term with constant viscosity on a curved sigma map:
# v* = v + dt (nu lap_phys(v) + g), lap_phys by finite differences.
# --------------------------------------------------------------------------
def test_predictor_viscous_term_sigma_map():
    """u, w quadratic in projected coordinates on the sigma map over a Gaussian
    bump (alpha, its derivatives, s_x and c0 all non-zero).  At particles with
    a complete all-fluid stencil, c_trans . D^v is the physical Laplacian of
    the field, so (v* - v)/dt = nu lap(v) + g.  A dropped factor 2 on the
    cross term, c0 on the wrong gradient component, or a wrong c3 changes it
    by O(1)."""
    d0, H = 0.01, 0.14
    bathy = S.Bathymetry(amp=[0.05], cx=[0.2], cy=[0.0], width=[0.07])
    nu = 2.0e-3
    sc = S.build_tank("pin_visc", 2, "SIGMA", 1.0, bathy,
                      dict(d0=d0, H=H, H_hat=H, nu_k=nu, smagorinsky=0, alpha_min=0.5,
                           alpha_max=4.0, gamma_over_dt=0.0), 0.4, jitter=0.0)
    xh, met, row, col = _csr(sc)
    f = sc.type == S.FLUID
    cu = dict(x=0.3, z=-0.4, xx=1.7, zz=-2.3, xz=3.1)
    cw = dict(x=-0.2, z=0.5, xx=-1.1, zz=0.8, xz=-2.6)

    def quad(c, X, Z):
        return (c["x"] * X + c["z"] * Z + 0.5 * c["xx"] * X * X + 0.5 * c["zz"] * Z * Z
                + c["xz"] * X * Z)

    X, Z = xh
    sc.u[f] = quad(cu, X[f], Z[f])
    sc.w[f] = quad(cw, X[f], Z[f])
    _, info = O.step(sc, probe=True)
    assert info["rc"] == 0
    sel = _full_fluid(sc, row, col, 20)
    assert sel.sum() > 100

    def phys(c, x, z):
        zh, _ = O.map_metric(sc, x, np.zeros_like(x), z)
        return quad(c, x, zh)

    h = 1e-3
    x, z = sc.x[sel], sc.z[sel]

    def lap_fd(c):
        fx = lambda s: phys(c, x + s * h, z)
        fz = lambda s: phys(c, x, z + s * h)
        d2 = lambda f: (-f(2) + 16 * f(1) - 30 * f(0) + 16 * f(-1) - f(-2)) / (12 * h * h)
        return d2(fx) + d2(fz)

    dt, g = sc.params["dt"], sc.params["g"]
    acc_u = (info["vstar"][0, sel] - sc.u[sel]) / dt
    acc_w = (info["vstar"][1, sel] - sc.w[sel]) / dt + g
    ref_u, ref_w = nu * lap_fd(cu), nu * lap_fd(cw)
    # the map's curvature terms must actually contribute
    assert np.abs(met[sel, 3]).max() > 0.1 and np.abs(met[sel, 1]).max() > 0.05
    assert np.allclose(acc_u, ref_u, rtol=0, atol=1e-6 * np.abs(ref_u).max())
    assert np.allclose(acc_w, ref_w, rtol=0, atol=1e-6 * np.abs(ref_w).max())


# --------------------------------------------------------------------------
# Variable viscosity: u = a (z - z0)^2 / 2 with the Smagorinsky model, so
# nu_E = (C_s r_e)^2 a (z - z0) is linear and
#   acc_x = nu a + (C_s r_e)^2 a^2 (z - z0),  acc_z = -g.
# --------------------------------------------------------------------------
def test_predictor_variable_viscosity_term():
    """BF map over a 1:10 slope, regular projected lattice (the free surface is
    placed a whole number of spacings above the bottom).  u_z = a (z - z0),
    so sqrt(2 S:S) = a (z - z0) and grad nu = (0, (C_s r_e)^2 a) in physical
    coordinates.  The second predictor term is then [(grad v) + (grad v)^T]
    grad nu = ((C_s r_e)^2 a^2 (z - z0), 0).  A transposed product, the
    projected instead of the physical gradient of nu, or S:S without its 1/2
    each change it."""
    d0 = 0.01
    slope = 0.1
    bathy = S.Bathymetry(h0=0.0, slope_x=slope)
    prm = dict(d0=d0, H=0.2, H_hat=0.2, nu_k=1.0e-4, smagorinsky=1, cs=0.2, gamma_over_dt=0.0)
    sc = S.build_tank("pin_varnu", 2, "BF", 1.0, bathy, prm, 0.4, jitter=0.0,
                      surface=lambda x, y: bathy.height(x, y) + 14 * d0)
    xh, met, row, col = _csr(sc)
    f = sc.type == S.FLUID
    a, z0 = 3.0, -0.2
    sc.u[f] = 0.5 * a * (sc.z[f] - z0) ** 2
    _, info = O.step(sc, probe=True)
    assert info["rc"] == 0
    full = _full_fluid(sc, row, col, 20)
    deep = _all_nb(row, col, full, full)
    assert deep.sum() > 50
    _, re, _ = O.radii(sc)
    K = (sc.params["cs"] * re) ** 2
    zr = sc.z[deep] - z0
    # the eddy viscosity itself (f_s = 1 away from walls)
    assert np.allclose(info["nu"][deep], sc.params["nu_k"] + K * a * zr, rtol=1e-9, atol=0)
    nu_i = sc.params["nu_k"] + K * a * zr
    dt, g = sc.params["dt"], sc.params["g"]
    acc_u = (info["vstar"][0, deep] - sc.u[deep]) / dt
    acc_w = (info["vstar"][1, deep] - sc.w[deep]) / dt + g
    ref_u = nu_i * a + K * a * a * zr
    assert np.abs(met[deep, 1]).min() > 0.05         # s_x = -h_x enters the Jacobian
    assert np.allclose(acc_u, ref_u, rtol=1e-8, atol=0)
    assert np.abs(acc_w).max() < 1e-8 * np.abs(ref_u).max()


# --------------------------------------------------------------------------
# Smagorinsky with the wall damping of Sec. 3.4 on a linear shear.
# --------------------------------------------------------------------------
def test_smagorinsky_linear_shear_and_wall_damping():
    """u = a (z - h0) over a flat bottom (zero at the bottom wall, as no-slip
    sets it), so sqrt(2 S:S) = |a| exactly at every particle the side walls do
    not see.  nu = nu_K + (C_s f_s r_e)^2 |a| with
    f_s = 1 - exp(-10 d0/d_s d_wall/r_e), d_wall the distance to the nearest
    wall neighbour, f_s = 1 without one.  d_s = 2 d0 separates d0/d_s from
    its inverse."""
    d0, h0 = 0.01, 0.02
    bathy = S.Bathymetry(h0=h0)
    prm = dict(d0=d0, H=0.1 + h0, H_hat=0.1, nu_k=1.0e-6, smagorinsky=1, cs=0.17, ds=0.02,
               gamma_over_dt=0.0)
    sc = S.build_tank("pin_smag", 2, "BF", 1.0, bathy, prm, 0.3, jitter=0.0)
    xh, met, row, col = _csr(sc)
    f = sc.type == S.FLUID
    a = -2.5
    sc.u[f] = a * (sc.z[f] - h0)
    _, info = O.step(sc, probe=True)
    assert info["rc"] == 0
    wall = sc.type == S.WALL
    bottom_wall = wall & (np.abs(sc.z - h0) < 1e-12)
    ok = np.zeros(sc.n, dtype=bool)
    dwall = np.full(sc.n, np.inf)
    for i in np.flatnonzero(f):
        nb = col[row[i]:row[i + 1]]
        if np.any(wall[nb] & ~bottom_wall[nb]):
            continue
        ok[i] = True
        wb = nb[wall[nb]]
        if wb.size:
            dwall[i] = np.sqrt((sc.x[wb] - sc.x[i]) ** 2 + (sc.z[wb] - sc.z[i]) ** 2).min()
    _, re, _ = O.radii(sc)
    fs = np.where(np.isfinite(dwall), 1.0 - np.exp(-10.0 * d0 / prm["ds"] * dwall / re), 1.0)
    ref = prm["nu_k"] + (prm["cs"] * fs * re) ** 2 * abs(a)
    near = ok & np.isfinite(dwall)
    assert near.sum() > 10 and (ok & ~near).sum() > 10
    assert np.allclose(info["nu"][ok], ref[ok], rtol=1e-9, atol=0)


# --------------------------------------------------------------------------
# Pressure right side: divergence of a linear v* and the stabilisation source.
# --------------------------------------------------------------------------
def _linear_velocity_tank(gamma_over_dt):
    d0 = 0.01
    bathy = S.Bathymetry(h0=0.0, slope_x=0.15)
    prm = dict(d0=d0, H=0.16, H_hat=0.16, nu_k=1.0e-3, smagorinsky=0,
               gamma_over_dt=gamma_over_dt)
    sc = S.build_tank("pin_div", 2, "BF", 1.0, bathy, prm, 0.4, jitter=0.1, seed=4)
    f = sc.type == S.FLUID
    A = np.array([[0.7, -1.3], [2.1, 0.4]])        # not symmetric, trace 1.1
    sc.u[f] = 0.05 + A[0, 0] * sc.x[f] + A[0, 1] * sc.z[f]
    sc.w[f] = -0.02 + A[1, 0] * sc.x[f] + A[1, 1] * sc.z[f]
    return sc, A


def _rows_without_wall_influence(sc, row, col, unk):
    """Rows that see no wall particle, and whose neighbours see none either
    (their v* is then the linear field plus dt g: D of a linear field is 0)."""
    wall = sc.type == S.WALL
    nowall = np.zeros(sc.n, dtype=bool)
    for i in range(sc.n):
        nowall[i] = not np.any(wall[col[row[i]:row[i + 1]]])
    f = sc.type == S.FLUID
    return _all_nb(row, col, nowall & f | (sc.type == S.VIRTUAL), unk & nowall)


def test_ppe_rhs_divergence_of_linear_vstar():
    """v = A r + c in physical coordinates on a jittered BF tank over a slope:
    v* = v + dt g is linear, its corrected projected gradient is exact and
    tr(J <grad^ (x) v*>) = tr(A).  With gamma = 0 the right side is
    rho/dt tr(A).  A transposed Jacobian (s_x on the wrong entry) or a missing
    rho/dt fails."""
    sc, A = _linear_velocity_tank(0.0)
    xh, met, row, col = _csr(sc)
    _, info = O.step(sc, probe=True)
    assert info["rc"] == 0
    unk = (sc.type == S.FLUID) & (info["fs"] == 0)
    sel = _rows_without_wall_influence(sc, row, col, unk)
    assert sel.sum() > 50
    ref = sc.params["rho"] / sc.params["dt"] * np.trace(A)
    assert np.allclose(info["ppe_b"][sel], ref, rtol=1e-10, atol=0)


def test_ppe_rhs_stabilisation_source():
    """The same linear field with gamma = 100 dt: the right side gains
    gamma (rho Jbar_i/J_i - rho^_i)/dt^2 (BF: J = 1, Jbar from the state), with
    rho^_i = rho sum_j V0 w_ij (self term included, all particle types) summed
    here by brute force from the kernel values.  A sign flip or a dropped self
    term fails."""
    sc, A = _linear_velocity_tank(100.0)
    xh, met, row, col = _csr(sc)
    _, info = O.step(sc, probe=True)
    assert info["rc"] == 0
    unk = (sc.type == S.FLUID) & (info["fs"] == 0)
    sel = _rows_without_wall_influence(sc, row, col, unk)
    l, re, _ = O.radii(sc)
    V0 = sc.params["d0"] ** 2
    rho = sc.params["rho"]
    X = xh.T
    rho_hat = np.empty(sc.n)
    for i in np.flatnonzero(sel):
        r = np.sqrt(((X - X[i]) ** 2).sum(axis=1))
        w, _ = O.kernel(2, l, r[r < re])
        rho_hat[i] = rho * V0 * w.sum()            # includes j = i (r = 0)
    dt = sc.params["dt"]
    gamma = 100.0 * dt
    target = rho * np.where(sc.jbar > 0, sc.jbar, 1.0)[sel] / met[sel, 0]
    ref = rho / dt * np.trace(A) + gamma * (target - rho_hat[sel]) / dt ** 2
    assert np.abs(target - rho_hat[sel]).max() > 1.0    # the jitter makes the source non-trivial
    assert np.allclose(info["ppe_b"][sel], ref, rtol=1e-10, atol=1e-9 * np.abs(ref).max())


def test_ppe_rhs_volume_ratio_sigma():
    """Sigma map, still fluid with an uneven Jbar: v* = dt g is uniform, so the
    divergence vanishes and the right side is gamma (rho Jbar/J - rho^)/dt^2
    with the Jbar the step used after its smoothing (Condition C of Sec. 3.6)
    and J = alpha from the map.  Inverting Jbar/J fails."""
    d0 = 0.01
    bathy = S.Bathymetry(amp=[0.04], cx=[0.15], cy=[0.0], width=[0.05])
    prm = dict(d0=d0, H=0.1, H_hat=0.1, smagorinsky=0, gamma_over_dt=100.0)
    sc = S.build_tank("pin_jbar", 2, "SIGMA", 1.0, bathy, prm, 0.3, jitter=0.0)
    xh, met, row, col = _csr(sc)
    f = sc.type == S.FLUID
    rng = np.random.default_rng(6)
    sc.jbar[:] = met[:, 0] * rng.uniform(0.9, 1.1, sc.n)
    _, info = O.step(sc, probe=True)
    assert info["rc"] == 0
    wall = sc.type == S.WALL
    unk = f & (info["fs"] == 0)
    sel = np.array([unk[i] and not np.any(wall[col[row[i]:row[i + 1]]]) for i in range(sc.n)])
    assert sel.sum() > 50
    l, re, _ = O.radii(sc)
    V0, rho, dt = d0 ** 2, sc.params["rho"], sc.params["dt"]
    X = xh.T
    ref = np.empty(sc.n)
    for i in np.flatnonzero(sel):
        r = np.sqrt(((X - X[i]) ** 2).sum(axis=1))
        w, _ = O.kernel(2, l, r[r < re])
        ref[i] = 100.0 * dt * (rho * info["jbar_used"][i] / met[i, 0] - rho * V0 * w.sum()) / dt ** 2
    ratio = info["jbar_used"][sel] / met[sel, 0]
    assert np.abs(ratio - 1.0).max() > 1e-3
    assert np.allclose(info["ppe_b"][sel], ref[sel], rtol=1e-9, atol=1e-9 * np.abs(ref[sel]).max())
