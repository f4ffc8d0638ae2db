"""Seeded synthetic scenarios: particle layouts, bathymetries and parameter sets.

This module only builds INPUTS.  It holds none of the solver's arithmetic
(no kernel, no SPH sums, no metric terms, no pressure equation); both the
CUDA library and the CPU oracle recompute the vertical map from the
bathymetry parameters on their own side.

Layout (projected space, Sec. 2.1): fluid particles sit on a lattice of
spacing d0 in the projected coordinates, at x^ = i*d0 (and y^ = j*d0 in 3-D);
each column holds nz = round(z^_top / d0) layers at z^ = k * z^_top / nz,
k = 1..nz, so the top layer lies on the free surface z^_top and the vertical
spacing is within d0/(2 nz) of d0.  Wall particles (type 1) form one layer on
each wall surface and virtual particles (type 2) two more layers outside
(Sec. 3.5, Fig. "two types of particles").  Fluid particles are jittered by
a uniform offset in [-jitter, +jitter]*d0 per projected coordinate.

Placing the lattice in physical space needs the vertical stretch of each
column: a column with bottom elevation h and layer stretch a has its k-th
layer at z = h + k*d0/a.  The stretch a per map kind is the scenario's
geometric choice of vertical particle spacing (E/BFE: a constant aspect
ratio; BF: 1; sigma: a fixed number of layers between bottom and still
water level, clamped).  This placement is the only place the layout touches
the map's definition, and neither side of the parity tests reads it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FLUID, WALL, VIRTUAL = 0, 1, 2
MAP_KINDS = {"E": 0, "BF": 1, "BFE": 2, "SIGMA": 3}

DEFAULT_PARAMS = dict(
    rho=1000.0,          # kg/m^3
    nu_k=1.0e-6,         # m^2/s kinematic viscosity
    g=9.81,              # m/s^2
    dt=1.0e-3,           # s
    d0=0.01,             # m, initial (projected) particle spacing
    l_over_d0=1.2,       # smoothing length l = 1.2 d0 (Sec. 3.1)
    re_over_l=2.0,       # effective radius r_e = 2 l (cubic spline support)
    gamma_over_dt=100.0, # stabilisation gamma = 100 dt (Sec. 3.3)
    cv_over_dt=100.0,    # volume smoothing C_V = 100 dt (Sec. 4.4.2)
    cs=0.2,              # Smagorinsky constant (Sec. 3.4)
    ds=0.01,             # reference spacing of the wall damping, 1 cm
    H=0.2,               # still-water level (physical)
    H_hat=0.2,           # projected column height of the sigma map
    alpha_min=1.0,       # sigma-map clamp range (Sec. 2.2.4)
    alpha_max=4.0,
    lam_fs_lo=0.2,       # free-surface eigenvalue thresholds
    lam_fs_hi=0.75,
    krylov_rtol=1.0e-9,
    krylov_max_iter=2000,
    smagorinsky=1,
    precision=0,         # 0 = FP64, 1 = mixed FP32 sums / FP64 solve
    volume_mode=2,       # 0 = Condition A, 1 = Condition B, 2 = Condition C
    ops_shift=0.0,       # particle regularisation, off unless a workload sets it
    ds_overlap=0.0,
    xsph_eps=0.0,
)

# Sec. 4.1: every simulation of the paper runs with optimized particle shifting
# (shift parameter 0.2), dynamic stabilization (40 % allowed overlap) and XSPH on
# free-surface particles (5e-3).  The wave workloads use them.
REGULARISATION = dict(ops_shift=0.2, ds_overlap=0.4, xsph_eps=5.0e-3)


@dataclass
class Bathymetry:
    """h(x,y) = h0 + sx*x + sy*y + cos_amp*cos(2 pi x / cos_len)
    + sum_g amp_g * exp(-((x-cx_g)^2 + (y-cy_g)^2) / (2 width_g^2))."""
    h0: float = 0.0
    slope_x: float = 0.0
    slope_y: float = 0.0
    cos_amp: float = 0.0
    cos_len: float = 1.0
    amp: list = field(default_factory=list)
    cx: list = field(default_factory=list)
    cy: list = field(default_factory=list)
    width: list = field(default_factory=list)

    def height(self, x, y=0.0):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        h = self.h0 + self.slope_x * x + self.slope_y * y
        if self.cos_amp != 0.0:
            h = h + self.cos_amp * np.cos(2.0 * math.pi * x / self.cos_len)
        for a, cx, cy, s in zip(self.amp, self.cx, self.cy, self.width):
            h = h + a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2.0 * s * s))
        return h


@dataclass
class Scenario:
    name: str
    dim: int
    map_kind: str
    aspect: float
    bathy: Bathymetry
    params: dict
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    p: np.ndarray
    jbar: np.ndarray
    type: np.ndarray
    box_lo: tuple
    box_hi: tuple

    @property
    def n(self):
        return int(self.x.shape[0])

    @property
    def n_fluid(self):
        return int(np.count_nonzero(self.type == FLUID))

    def copy(self):
        c = Scenario(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        for k in ("x", "y", "z", "u", "v", "w", "p", "jbar", "type"):
            setattr(c, k, getattr(self, k).copy())
        c.params = dict(self.params)
        return c

    def state_arrays(self):
        return dict(x=self.x, y=self.y, z=self.z, u=self.u, v=self.v, w=self.w,
                    p=self.p, jbar=self.jbar, type=self.type)


def _layer_stretch(kind, aspect, bathy, prm, x, y):
    """Vertical stretch a of the particle layers of a column (layer k sits at
    physical height base + k*d0/a) and the column's base elevation."""
    h = bathy.height(x, y)
    if kind == "E":
        return np.full_like(h, aspect), np.zeros_like(h)
    if kind == "BF":
        return np.ones_like(h), h
    if kind == "BFE":
        return np.full_like(h, aspect), h
    if kind == "SIGMA":
        depth = prm["H"] - h
        a = np.where(depth > 0, prm["H_hat"] / np.maximum(depth, 1e-300), prm["alpha_max"])
        return np.clip(a, prm["alpha_min"], prm["alpha_max"]), h
    raise ValueError(kind)


def build_tank(name, dim, kind, aspect, bathy, params, L, W=0.0, surface=None,
               velocity=None, seed=0, jitter=0.1, wall_extra_layers=4,
               box_top_margin=None, min_layers=1):
    """Fill a tank [0,L] (x [0,W] in 3-D) with fluid up to `surface(x, y)`
    (physical elevation) and surround it by wall + virtual layers."""
    prm = dict(DEFAULT_PARAMS)
    prm.update(params)
    d0 = prm["d0"]
    rng = np.random.default_rng(seed)
    nx = int(round(L / d0))
    ny = int(round(W / d0)) if dim == 3 else 0
    if surface is None:
        surface = lambda x, y: np.full_like(np.asarray(x, dtype=np.float64), prm["H"])

    # ---- fluid columns (projected lattice) ----
    ix = np.arange(1, nx)
    if dim == 3:
        iy = np.arange(1, ny)
        CX, CY = np.meshgrid(ix * d0, iy * d0, indexing="xy")
        colx, coly = CX.ravel(), CY.ravel()
    else:
        colx = ix * d0
        coly = np.zeros_like(colx)
    a_col, base_col = _layer_stretch(kind, aspect, bathy, prm, colx, coly)
    top_proj = a_col * (surface(colx, coly) - base_col)
    nz_col = np.maximum(np.rint(top_proj / d0).astype(np.int64), 0)
    nz_col[nz_col < min_layers] = 0   # columns too shallow for a moment matrix stay dry
    ncol = colx.shape[0]
    rep = nz_col
    fx = np.repeat(colx, rep)
    fy = np.repeat(coly, rep)
    fk = np.concatenate([np.arange(1, k + 1) for k in nz_col]) if ncol else np.zeros(0)
    # the nz layers of a column are spaced z^_top / nz (within d0/(2 nz) of d0):
    # the top layer lies on the free surface, so a flat physical surface stays
    # flat, and the lowest layer sits one spacing above the bottom wall
    sp = np.repeat(top_proj / np.maximum(nz_col, 1), rep)
    fzh = fk * sp
    nf = fx.shape[0]
    jx = rng.uniform(-jitter, jitter, nf) * d0
    jy = rng.uniform(-jitter, jitter, nf) * d0 if dim == 3 else np.zeros(nf)
    jz = rng.uniform(-jitter, jitter, nf) * d0
    fx = fx + jx
    fy = fy + jy
    fzh = fzh + jz
    a_f, base_f = _layer_stretch(kind, aspect, bathy, prm, fx, fy)
    fz = base_f + fzh / a_f
    # column top (un-jittered) -> hydrostatic initial pressure, zero on the top layer
    top_phys_col = base_col + top_proj / a_col
    top_f = np.repeat(top_phys_col, rep)

    # ---- walls ----
    nzw = int(nz_col.max() if ncol else 0) + wall_extra_layers
    wx, wy, wzh, wt = [], [], [], []

    def add(xs, ys, zhs, ts):
        wx.append(np.asarray(xs, dtype=np.float64).ravel())
        wy.append(np.asarray(ys, dtype=np.float64).ravel())
        wzh.append(np.asarray(zhs, dtype=np.float64).ravel())
        wt.append(np.asarray(ts, dtype=np.int32).ravel())

    bx = np.arange(-2, nx + 3)
    by = np.arange(-2, ny + 3) if dim == 3 else np.array([0])
    for kz in (0, -1, -2):  # bottom
        BX, BY = np.meshgrid(bx, by, indexing="xy")
        inside = (BX >= 0) & (BX <= nx)
        if dim == 3:
            inside &= (BY >= 0) & (BY <= ny)
        t = np.where((kz == 0) & inside, WALL, VIRTUAL)
        add(BX * d0, (BY * d0) if dim == 3 else np.zeros_like(BX, dtype=np.float64),
            np.full(BX.shape, kz * d0), t)
    kz = np.arange(1, nzw + 1)
    for side in ((0, -1, -2), (nx, nx + 1, nx + 2)):  # x walls
        for k, cx in enumerate(side):
            if dim == 3:
                BY, KZ = np.meshgrid(by, kz, indexing="xy")
                t = np.where((k == 0) & (BY >= 0) & (BY <= ny), WALL, VIRTUAL)
                add(np.full(BY.shape, cx * d0), BY * d0, KZ * d0, t)
            else:
                add(np.full(kz.shape, cx * d0), np.zeros(kz.shape), kz * d0,
                    np.full(kz.shape, WALL if k == 0 else VIRTUAL))
    if dim == 3:
        for side in ((0, -1, -2), (ny, ny + 1, ny + 2)):  # y walls
            for k, cy in enumerate(side):
                BX, KZ = np.meshgrid(np.arange(1, nx), kz, indexing="xy")
                t = np.full(BX.shape, WALL if k == 0 else VIRTUAL)
                add(BX * d0, np.full(BX.shape, cy * d0), KZ * d0, t)
    wx = np.concatenate(wx)
    wy = np.concatenate(wy)
    wzh = np.concatenate(wzh)
    wt = np.concatenate(wt)
    a_w, base_w = _layer_stretch(kind, aspect, bathy, prm, wx, wy)
    wz = base_w + wzh / a_w

    x = np.concatenate([fx, wx])
    y = np.concatenate([fy, wy]) if dim == 3 else np.zeros(nf + wx.shape[0])
    z = np.concatenate([fz, wz])
    typ = np.concatenate([np.full(nf, FLUID, dtype=np.int32), wt]).astype(np.int32)
    n = x.shape[0]
    u = np.zeros(n)
    v = np.zeros(n)
    w = np.zeros(n)
    if velocity is not None and nf:
        fu, fv, fw = velocity(fx, fy, fz)
        u[:nf], v[:nf], w[:nf] = fu, fv, fw
    p = np.zeros(n)
    p[:nf] = np.maximum(prm["rho"] * prm["g"] * (top_f - fz), 0.0)
    # Jbar carries each particle's initial volume (V_i = V0 J_i / Jbar_i, Sec. 3.6):
    # a fluid particle's lattice cell is d0^(d-1) x its column's layer spacing, so
    # Jbar0 = J0 * d0 / spacing (= J0 on an exact d0 lattice); walls and virtual
    # particles sit on the exact lattice (<= 0: the solver sets Jbar = J there).
    jbar = np.zeros(n)
    jbar[:nf] = a_f * d0 / sp

    zmax = float(wzh.max() if wzh.size else 0.0)
    if box_top_margin is None:
        box_top_margin = 0.5 * zmax + 10 * d0
    box_lo = (-3 * d0, -3 * d0 if dim == 3 else 0.0, -3 * d0)
    box_hi = (L + 3 * d0, (W + 3 * d0) if dim == 3 else 0.0, zmax + box_top_margin)
    return Scenario(name, dim, kind, float(aspect), bathy, prm, x, y, z, u, v, w, p,
                    jbar, typ, box_lo, box_hi)


def solitary_wave(amplitude, depth, x0, g):
    """First-order solitary wave: eta = A sech^2(k (x - x0)), k = sqrt(3A/(4 d^3)),
    depth-uniform horizontal velocity u = sqrt(g d) eta / d."""
    k = math.sqrt(3.0 * amplitude / (4.0 * depth ** 3))
    c = math.sqrt(g * depth)

    def eta(x):
        return amplitude / np.cosh(k * (np.asarray(x) - x0)) ** 2

    def vel(x, y, z):
        e = eta(x)
        return c * e / depth, np.zeros_like(e), np.zeros_like(e)

    return eta, vel


# ---------------------------------------------------------------------------
# The five workloads, plus small variants for the parity tests.
# ---------------------------------------------------------------------------

def still_water_bf(d0=0.01, L=1.0, H=0.2, seed=0, jitter=0.1, precision=0, **kw):
    """2-D BF-SPH still water over a 1:10 slope, mean depth 0.2 m:
    h(x) = 0.1 (x - 0.5), so the depth runs 0.25 m -> 0.15 m.  Particle
    regularisation on, as in every simulation of Sec. 4 (without it the
    jittered tank's motion grows until the run fails near step 85, in the
    oracle and the CUDA path alike)."""
    bathy = Bathymetry(h0=-0.05 * (L / 1.0), slope_x=0.1)
    prm = dict(d0=d0, H=H, H_hat=H, dt=1.0e-3, precision=precision)
    prm.update(REGULARISATION)
    prm.update(kw)
    return build_tank("still_water_bf", 2, "BF", 1.0, bathy, prm, L, seed=seed, jitter=jitter)


def solitary_sigma(d0=1.0 / 90.0, L=10.0, depth=0.5, bump=0.3, bump_x=5.0, bump_s=0.25,
                   wave=0.2, x0=2.0, seed=0, precision=1, jitter=0.0, **kw):
    """2-D sigma-SPH solitary wave (H/d = 0.2) over a Gaussian bump 0.3 m high,
    1 m wide (+-2 s), in a 10 m channel of depth 0.5 m; alpha = 1..2.5."""
    bathy = Bathymetry(amp=[bump], cx=[bump_x], cy=[0.0], width=[bump_s])
    prm = dict(d0=d0, H=depth, H_hat=depth, dt=1.0e-3, precision=precision,
               alpha_min=1.0, alpha_max=4.0)
    prm.update(REGULARISATION)
    prm.update(kw)
    eta, vel = solitary_wave(wave * depth, depth, x0, prm.get("g", 9.81))
    surf = lambda x, y: depth + eta(x)
    return build_tank("solitary_sigma", 2, "SIGMA", 1.0, bathy, prm, L, surface=surf,
                      velocity=vel, seed=seed, jitter=jitter)


def beach_bfe_3d(d0=0.043, L=20.0, W=4.0, depth=1.0, slope=0.05, aspect=4.0, wave=0.1,
                 x0=3.0, seed=0, precision=1, jitter=0.0, **kw):
    """3-D BFE-SPH solitary wave on a 1:20 beach, 20 x 4 m basin, depth 1 m -> 0,
    ellipsoidal particles with aspect ratio 4, on a regular projected lattice
    (a random jitter's density errors drive the stabilisation term of the
    pressure equation hard at this aspect ratio).  Columns with fewer than
    three projected layers are left dry (a one- or two-layer wedge has no
    moment matrix).  Particle regularisation is on (Sec. 4.1).  The
    Smagorinsky model is off: at aspect 4 its eddy viscosity, applied through
    the explicit viscous term with the ill-conditioned SPH(2) second
    derivatives of free-surface particles, grows without bound within a few
    steps (both the CUDA path and the oracle)."""
    bathy = Bathymetry(slope_x=slope)
    prm = dict(d0=d0, H=depth, H_hat=depth * aspect, dt=1.0e-3, precision=precision,
               smagorinsky=0)
    prm.update(REGULARISATION)
    prm.update(kw)
    eta, vel = solitary_wave(wave, depth, x0, prm.get("g", 9.81))
    surf = lambda x, y: depth + eta(x)
    return build_tank("beach_bfe_3d", 3, "BFE", aspect, bathy, prm, L, W, surface=surf,
                      velocity=vel, seed=seed, min_layers=3, jitter=jitter)


def random_bumps(rng, n, amp_lo, amp_hi, x_lo, x_hi, width, depth, min_depth):
    while True:
        amp = rng.uniform(amp_lo, amp_hi, n)
        cx = rng.uniform(x_lo, x_hi, n)
        b = Bathymetry(amp=list(amp), cx=list(cx), cy=[0.0] * n, width=[width] * n)
        xs = np.linspace(0.0, x_hi + x_lo, 4001)
        if depth - b.height(xs).max() >= min_depth:
            return b


def adjoint_sigma(d0=0.01, L=10.0, depth=0.5, n_bumps=16, wave=0.1, x0=3.0, seed=1,
                  precision=0, **kw):
    """2-D sigma-SPH with flat 0.5 m + 16 random Gaussian bumps (seed 1)."""
    rng = np.random.default_rng(seed)
    bathy = random_bumps(rng, n_bumps, 0.02, 0.10, 1.0, 9.0, 0.2, depth, 0.15)
    prm = dict(d0=d0, H=depth, H_hat=depth, dt=1.0e-3, precision=precision)
    prm.update(kw)
    eta, vel = solitary_wave(wave, depth, x0, prm.get("g", 9.81))
    surf = lambda x, y: depth + eta(x)
    return build_tank("adjoint_sigma", 2, "SIGMA", 1.0, bathy, prm, L, surface=surf,
                      velocity=vel, seed=seed)


def ensemble_sizes(n_scen=64, lo=5e3, hi=2e5, seed=2):
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(v))) for v in rng.uniform(math.log(lo), math.log(hi), n_scen)]


def ensemble(n_scen=64, seed=2, precision=1, jitter=0.0, **kw):
    """64 2-D sigma scenarios, particle counts log-uniform 5e3..2e5 (seed 2),
    d0 = sqrt(5 / N_s) on a 10 m x 0.5 m projected channel, 4 random bumps each,
    regular projected lattice and particle regularisation as the solitary wave."""
    sizes = ensemble_sizes(n_scen, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    out = []
    for s, ns in enumerate(sizes):
        d0 = math.sqrt(5.0 / ns)
        bathy = random_bumps(rng, 4, 0.02, 0.2, 1.0, 9.0, 0.25, 0.5, 0.2)
        prm = dict(d0=d0, H=0.5, H_hat=0.5, dt=1.0e-3, precision=precision)
        prm.update(REGULARISATION)
        prm.update(kw)
        eta, vel = solitary_wave(0.05, 0.5, 2.0, 9.81)
        out.append(build_tank(f"ensemble_{s}", 2, "SIGMA", 1.0, bathy, prm, 10.0,
                              surface=lambda x, y: 0.5 + eta(x), velocity=vel, seed=seed + s,
                              jitter=jitter))
    return out


def efficiency_tank(kind, precision=1, **kw):
    """The hydrostatic tank of the BF / BFE / sigma efficiency comparison
    (Sec. 4.4.1, Table fig:s4_s_time), with a stated stand-in for the bottom of
    the missing figure: 1 m long, still-water level H = 0.2 m, bottom
    h(x) = 0.12 x + 0.01 (1 - cos(2 pi x / 0.5)) -- a slope plus a sine, depth
    0.2 m at x = 0 and 0.08 m at the shallowest point x = 1 m.  The models share
    the vertical spacing at the shallowest point (0.2 cm): BF with d0 = 0.2 cm,
    BFE with d0 = 0.5 cm and alpha = 2.5, sigma with d0 = 0.5 cm and
    H = H^ = 0.2 m (alpha = 1 at the deepest point, 2.5 at the shallowest).
    Regular lattice, hydrostatic start, dt = 5e-4 s, particle regularisation on
    (Sec. 4)."""
    bathy = Bathymetry(slope_x=0.12, h0=0.01, cos_amp=-0.01, cos_len=0.5)
    d0 = 0.002 if kind == "BF" else 0.005
    aspect = 2.5 if kind == "BFE" else 1.0
    prm = dict(d0=d0, H=0.2, H_hat=0.2 * aspect if kind != "SIGMA" else 0.2, dt=5.0e-4,
               precision=precision, alpha_min=1.0, alpha_max=2.5)
    prm.update(REGULARISATION)
    prm.update(kw)
    return build_tank(f"efficiency_{kind.lower()}", 2, kind, aspect, bathy, prm, 1.0, jitter=0.0)


def dam_break_sigma_3d(d0=0.0025, x_dam=0.08, precision=1, **kw):
    """3-D sigma-SPH dam break (Sec. 4.4.3): bottom h(x, y) = 0.1 x + 2 cos(2 pi x / 20)
    in cm (here h = 0.1 x + 0.02 cos(2 pi x / 0.2) m), projected domain 25 x 20 x 10 cm,
    H = 15 cm, H^ = 10 cm (alpha = H^/(H - h), 0.63-0.91), d0 = 0.25 cm, dt = 1e-4 s,
    Condition C with C_V = 100 dt.  The figure with the dam's position is missing:
    the water column stands at the still-water level H over 0 <= x < x_dam (8 cm),
    the rest of the basin is dry.  Particle regularisation on (Sec. 4)."""
    bathy = Bathymetry(slope_x=0.1, cos_amp=0.02, cos_len=0.2)
    prm = dict(d0=d0, H=0.15, H_hat=0.10, dt=1.0e-4, precision=precision,
               alpha_min=0.5, alpha_max=1.5, volume_mode=2)
    prm.update(REGULARISATION)
    prm.update(kw)
    H = prm["H"]
    surf = lambda x, y: np.where(np.asarray(x) < x_dam, H, bathy.height(x, y))  # noqa: E731
    return build_tank("dam_break_sigma_3d", 3, "SIGMA", 1.0, bathy, prm, 0.25, 0.20,
                      surface=surf, jitter=0.0)


def small_tank(dim=2, kind="BF", L=0.3, W=0.1, H=0.1, d0=0.01, seed=0, aspect=1.0,
               bathy=None, jitter=0.1, with_wave=False, precision=0, **kw):
    """A few-thousand-particle tank for parity and edge-case tests."""
    if bathy is None:
        bathy = Bathymetry(amp=[0.3 * H], cx=[0.5 * L], cy=[0.5 * W], width=[0.15 * L])
    prm = dict(d0=d0, H=H, H_hat=H if kind != "BFE" else H * aspect, dt=1.0e-3,
               precision=precision)
    if kind == "E":
        prm["H_hat"] = H * aspect
    prm.update(kw)
    surf = None
    vel = None
    if with_wave:
        eta, vel = solitary_wave(0.2 * H, H, 0.3 * L, prm.get("g", 9.81))
        surf = lambda x, y: H + eta(x)
    return build_tank(f"small_{dim}d_{kind}", dim, kind, aspect, bathy, prm, L,
                      W if dim == 3 else 0.0, surface=surf, velocity=vel, seed=seed,
                      jitter=jitter)
