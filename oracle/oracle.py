"""ctypes front end of the plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.  Arrays are numpy float64 / int32, component-major.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAP = {"E": 0, "BF": 1, "BFE": 2, "SIGMA": 3}
_lib = None


class OrcBathy(C.Structure):
    _fields_ = [("h0", C.c_double), ("slope_x", C.c_double), ("slope_y", C.c_double),
                ("cos_amp", C.c_double), ("cos_len", C.c_double), ("n_gauss", C.c_int),
                ("pad_", C.c_int), ("amp", C.POINTER(C.c_double)), ("cx", C.POINTER(C.c_double)),
                ("cy", C.POINTER(C.c_double)), ("width", C.POINTER(C.c_double))]


class OrcParams(C.Structure):
    _fields_ = [("dim", C.c_int), ("map_kind", C.c_int), ("aspect", C.c_double)] + [
        (k, C.c_double) for k in ("rho", "nu_k", "g", "dt", "d0", "l_over_d0", "re_over_l",
                                  "gamma_over_dt", "cv_over_dt", "cs", "ds", "H", "H_hat",
                                  "alpha_min", "alpha_max", "lam_fs_lo", "lam_fs_hi",
                                  "ppe_rtol")] + [
        (k, C.c_int) for k in ("ppe_max_iter", "smagorinsky", "volume_mode", "neighbour_mode",
                               "smoothing_mode", "pad_")] + [
        (k, C.c_double) for k in ("ops_shift", "ds_overlap", "xsph_eps")] + [
        ("operators", C.c_int), ("wall_slip", C.c_int)]


class OrcState(C.Structure):
    _fields_ = [("n", C.c_int), ("pad_", C.c_int)] + [
        (k, C.POINTER(C.c_double)) for k in ("x", "y", "z", "u", "v", "w", "p", "jbar")] + [
        ("type", C.POINTER(C.c_int32))]


class OrcProbe(C.Structure):
    _fields_ = [("fs", C.POINTER(C.c_int32)), ("rho_hat", C.POINTER(C.c_double)),
                ("nu", C.POINTER(C.c_double)), ("lam_min", C.POINTER(C.c_double)),
                ("vstar", C.POINTER(C.c_double)), ("ppe_b", C.POINTER(C.c_double)),
                ("x_test", C.POINTER(C.c_double)), ("ppe_Ax", C.POINTER(C.c_double)),
                ("jbar_used", C.POINTER(C.c_double)), ("n_iter", C.c_int), ("pad_", C.c_int),
                ("resid", C.c_double), ("vwall", C.POINTER(C.c_double))]


def lib():
    global _lib
    if _lib is None:
        # VCT_ORACLE_LIB names a separately built copy of the oracle (the planted-
        # mistake tests compile mutated copies and run the pins against them)
        path = os.environ.get("VCT_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.orc_kernel.argtypes = [C.c_int, C.c_double, C.c_int, dp, dp, dp]
        L.orc_map_coeffs.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcBathy), C.c_int, dp, dp, dp]
        L.orc_map.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcBathy), C.c_int, dp, dp, dp, dp, dp]
        L.orc_neighbours.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_int,
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.c_int64]
        L.orc_neighbours.restype = C.c_int64
        L.orc_sph2_derivatives.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcBathy),
                                           C.POINTER(OrcState), dp, C.c_int, dp, dp, dp]
        L.orc_summation_gradient.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcBathy),
                                             C.POINTER(OrcState), dp, C.c_int, dp]
        L.orc_moment_matrices.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcBathy),
                                          C.POINTER(OrcState), dp]
        L.orc_volume_smoothing.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcBathy),
                                           C.POINTER(OrcState), C.c_int]
        L.orc_step.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcBathy), C.POINTER(OrcState),
                               C.c_int, C.POINTER(OrcProbe), C.POINTER(C.c_int)]
        L.orc_regularise.argtypes = [C.POINTER(OrcParams), C.POINTER(OrcBathy),
                                     C.POINTER(OrcState), C.POINTER(C.c_int32)]
        L.orc_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def set_threads(n):
    return lib().orc_set_threads(int(n))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Keep:
    """Holds the numpy buffers a ctypes struct points into."""

    def __init__(self):
        self.refs = []

    def f64(self, a):
        a = _f64(a)
        self.refs.append(a)
        return a


def make_bathy(b, keep):
    amp = keep.f64(np.asarray(b.amp, dtype=np.float64).reshape(-1) if len(b.amp) else np.zeros(1))
    cx = keep.f64(np.asarray(b.cx, dtype=np.float64) if len(b.cx) else np.zeros(1))
    cy = keep.f64(np.asarray(b.cy, dtype=np.float64) if len(b.cy) else np.zeros(1))
    wd = keep.f64(np.asarray(b.width, dtype=np.float64) if len(b.width) else np.ones(1))
    return OrcBathy(b.h0, b.slope_x, b.slope_y, b.cos_amp, b.cos_len, len(b.amp), 0,
                    _dp(amp), _dp(cx), _dp(cy), _dp(wd))


def make_params(sc, neighbour_mode=1, smoothing_mode=1, rtol=1e-13, max_iter=20000, **over):
    p = dict(sc.params)
    p.update(over)
    P = OrcParams()
    P.dim = sc.dim
    P.map_kind = MAP[sc.map_kind]
    P.aspect = sc.aspect
    for k in ("rho", "nu_k", "g", "dt", "d0", "l_over_d0", "re_over_l", "gamma_over_dt",
              "cv_over_dt", "cs", "ds", "H", "H_hat", "alpha_min", "alpha_max", "lam_fs_lo",
              "lam_fs_hi"):
        setattr(P, k, float(p[k]))
    P.ppe_rtol = float(p.get("oracle_rtol", rtol))
    P.ppe_max_iter = int(p.get("oracle_max_iter", max_iter))
    P.smagorinsky = int(p["smagorinsky"])
    P.volume_mode = int(p["volume_mode"])
    P.neighbour_mode = int(neighbour_mode)
    P.smoothing_mode = int(smoothing_mode)
    for k in ("ops_shift", "ds_overlap", "xsph_eps"):
        setattr(P, k, float(p.get(k, 0.0)))
    P.operators = int(p.get("operators", 0))
    P.wall_slip = int(p.get("wall_slip", 0))
    return P


class OracleState:
    """Copies of the scenario's state arrays that the oracle updates in place."""

    def __init__(self, sc):
        self.n = sc.n
        self.x = _f64(sc.x).copy()
        self.y = _f64(sc.y).copy()
        self.z = _f64(sc.z).copy()
        self.u = _f64(sc.u).copy()
        self.v = _f64(sc.v).copy()
        self.w = _f64(sc.w).copy()
        self.p = _f64(sc.p).copy()
        self.jbar = _f64(sc.jbar).copy()
        self.type = np.ascontiguousarray(sc.type, dtype=np.int32)

    def struct(self):
        return OrcState(self.n, 0, _dp(self.x), _dp(self.y), _dp(self.z), _dp(self.u),
                        _dp(self.v), _dp(self.w), _dp(self.p), _dp(self.jbar),
                        self.type.ctypes.data_as(C.POINTER(C.c_int32)))

    def arrays(self):
        return dict(x=self.x, y=self.y, z=self.z, u=self.u, v=self.v, w=self.w, p=self.p,
                    jbar=self.jbar, type=self.type)


def kernel(dim, l, r):
    r = _f64(r)
    w = np.zeros_like(r)
    dw = np.zeros_like(r)
    lib().orc_kernel(dim, l, r.size, _dp(r), _dp(w), _dp(dw))
    return w, dw


def map_coeffs(sc, x, y=None):
    keep = _Keep()
    x = keep.f64(x)
    y = keep.f64(np.zeros_like(x) if y is None else y)
    B = make_bathy(sc.bathy, keep)
    P = make_params(sc)
    ab = np.zeros((x.size, 10))
    lib().orc_map_coeffs(C.byref(P), C.byref(B), x.size, _dp(x), _dp(y), _dp(ab))
    return ab


def map_metric(sc, x, y, z):
    keep = _Keep()
    x, y, z = keep.f64(x), keep.f64(y), keep.f64(z)
    B = make_bathy(sc.bathy, keep)
    P = make_params(sc)
    zh = np.zeros_like(x)
    met = np.zeros((x.size, 7))
    lib().orc_map(C.byref(P), C.byref(B), x.size, _dp(x), _dp(y), _dp(z), _dp(zh), _dp(met))
    return zh, met


def radii(sc):
    p = sc.params
    l = p["l_over_d0"] * p["d0"]
    re = p["re_over_l"] * l
    return l, re, re * re


def projected(sc, x=None, y=None, z=None):
    x = sc.x if x is None else x
    y = sc.y if y is None else y
    z = sc.z if z is None else z
    zh, met = map_metric(sc, x, y, z)
    if sc.dim == 2:
        return np.stack([_f64(x), zh]), met
    return np.stack([_f64(x), _f64(y), zh]), met


def neighbours(dim, xh_soa, re, re2, mode=0):
    xh = np.ascontiguousarray(xh_soa, dtype=np.float64)
    n = xh.shape[1]
    row = np.zeros(n + 1, dtype=np.int64)
    nnz = lib().orc_neighbours(dim, n, _dp(xh), re, re2, mode,
                               row.ctypes.data_as(C.POINTER(C.c_int64)), None, 0)
    if nnz < 0:
        nnz = int(row[-1])
    col = np.zeros(max(int(nnz), 1), dtype=np.int32)
    r = lib().orc_neighbours(dim, n, _dp(xh), re, re2, mode,
                             row.ctypes.data_as(C.POINTER(C.c_int64)),
                             col.ctypes.data_as(C.POINTER(C.c_int32)), col.size)
    assert r == nnz
    return row, col[:nnz]


def sph2_derivatives(sc, phi, state=None, **over):
    """phi: (ncomp, n).  Returns grad_hat (ncomp, d, n), d2_hat (ncomp, m, n),
    lap_phys (ncomp, n)."""
    keep = _Keep()
    st = OracleState(sc) if state is None else state
    B = make_bathy(sc.bathy, keep)
    P = make_params(sc, **over)
    phi = keep.f64(np.atleast_2d(phi))
    nc = phi.shape[0]
    d = sc.dim
    m = 3 if d == 2 else 6
    g = np.zeros((nc, d, sc.n))
    d2 = np.zeros((nc, m, sc.n))
    lap = np.zeros((nc, sc.n))
    S = st.struct()
    rc = lib().orc_sph2_derivatives(C.byref(P), C.byref(B), C.byref(S), _dp(phi), nc, _dp(g),
                                    _dp(d2), _dp(lap))
    if rc:
        raise RuntimeError(f"oracle sph2_derivatives failed: {rc}")
    return g, d2, lap


def summation_gradient(sc, phi, **over):
    """The summation gradient of Eq. (gra_sum), projected coordinates:
    (ncomp, d, n) for phi (ncomp, n)."""
    keep = _Keep()
    st = OracleState(sc)
    B = make_bathy(sc.bathy, keep)
    P = make_params(sc, **over)
    phi = keep.f64(np.atleast_2d(phi))
    nc = phi.shape[0]
    out = np.zeros((nc, sc.dim, sc.n))
    S = st.struct()
    rc = lib().orc_summation_gradient(C.byref(P), C.byref(B), C.byref(S), _dp(phi), nc, _dp(out))
    if rc:
        raise RuntimeError(f"oracle summation_gradient failed: {rc}")
    return out


def moment_matrices(sc, **over):
    """The SPH(2) moment matrices M_i (n, m, m) of the scenario's state (zero
    for particles that are not fluid)."""
    keep = _Keep()
    st = OracleState(sc)
    B = make_bathy(sc.bathy, keep)
    P = make_params(sc, **over)
    m = 3 if sc.dim == 2 else 6
    M = np.zeros((sc.n, m, m))
    S = st.struct()
    rc = lib().orc_moment_matrices(C.byref(P), C.byref(B), C.byref(S), _dp(M))
    if rc:
        raise RuntimeError(f"oracle moment_matrices failed: {rc}")
    return M


def volume_smoothing(sc, state, mode):
    keep = _Keep()
    B = make_bathy(sc.bathy, keep)
    P = make_params(sc)
    S = state.struct()
    return lib().orc_volume_smoothing(C.byref(P), C.byref(B), C.byref(S), mode)


def regularise(sc, state, fs=None, **over):
    """Particle regularisation alone (dynamic stabilization, XSPH, shifting)
    on `state` in place, neighbour sets at its positions; fs: free-surface flags."""
    keep = _Keep()
    B = make_bathy(sc.bathy, keep)
    P = make_params(sc, **over)
    S = state.struct()
    f = None if fs is None else np.ascontiguousarray(fs, dtype=np.int32)
    return lib().orc_regularise(C.byref(P), C.byref(B), C.byref(S),
                                None if f is None else f.ctypes.data_as(C.POINTER(C.c_int32)))


def step(sc, state=None, nsteps=1, probe=False, x_test=None, **over):
    """Advance `state` (an OracleState; a fresh copy of the scenario if None) by
    nsteps.  Returns (state, info) where info holds the probe of the last step."""
    keep = _Keep()
    st = OracleState(sc) if state is None else state
    B = make_bathy(sc.bathy, keep)
    P = make_params(sc, **over)
    n, d = sc.n, sc.dim
    info = {}
    pr = None
    if probe:
        info = dict(fs=np.zeros(n, dtype=np.int32), rho_hat=np.zeros(n), nu=np.zeros(n),
                    lam_min=np.zeros(n), vstar=np.zeros((d, n)), ppe_b=np.zeros(n),
                    jbar_used=np.zeros(n), vwall=np.zeros((d, n)))
        xt = keep.f64(x_test) if x_test is not None else None
        if xt is not None:
            info["ppe_Ax"] = np.zeros(n)
        pr = OrcProbe(info["fs"].ctypes.data_as(C.POINTER(C.c_int32)), _dp(info["rho_hat"]),
                      _dp(info["nu"]), _dp(info["lam_min"]), _dp(info["vstar"]),
                      _dp(info["ppe_b"]), _dp(xt), _dp(info.get("ppe_Ax")),
                      _dp(info["jbar_used"]), 0, 0, 0.0, _dp(info["vwall"]))
    S = st.struct()
    iters = C.c_int(0)
    rc = lib().orc_step(C.byref(P), C.byref(B), C.byref(S), nsteps,
                        C.byref(pr) if pr is not None else None, C.byref(iters))
    info["rc"] = rc
    info["iters"] = iters.value
    if pr is not None:
        info["n_iter"] = pr.n_iter
        info["resid"] = pr.resid
    return st, info


def ppe_system(sc, **over):
    """The pressure equation of one step from the scenario's state (Sec. 3.3,
    Eqs. VCT_ppe and PNC) as a dense matrix on its unknown rows (fluid particles
    off the free surface), assembled column by column from the oracle's own
    operator application (the probe's A x for unit vectors x), with the step's
    right side b and solution p.  Returns (rows, A, b, p); rows are caller
    indices.  One oracle step per unknown: small cases only."""
    st, info = step(sc, probe=True, **over)
    fs = info["fs"]
    rows = np.flatnonzero((sc.type == 0) & (fs == 0))
    m = rows.size
    A = np.zeros((m, m))
    for k, col in enumerate(rows):
        e = np.zeros(sc.n)
        e[col] = 1.0
        _, ik = step(sc, probe=True, x_test=e, **over)
        A[:, k] = ik["ppe_Ax"][rows]
    return rows, A, info["ppe_b"][rows].copy(), st.p[rows].copy()


def ppe_adjoint(A, p_bar):
    """b_bar = A^-T p_bar: the adjoint of p = A^-1 b with respect to b (the
    transpose solve; numpy's dense LU)."""
    return np.linalg.solve(A.T, p_bar)


def _spline(q):
    """The cubic spline's shape (unnormalised): 1 - 1.5 q^2 + 0.75 q^3 below 1,
    0.25 (2 - q)^3 below 2, 0 beyond."""
    q = np.asarray(q, dtype=np.float64)
    return np.where(q < 1.0, 1.0 - 1.5 * q * q + 0.75 * q ** 3,
                    np.where(q < 2.0, 0.25 * (2.0 - q) ** 3, 0.0))


def gauge_levels(sc, fs, gauges, x=None, y=None, z=None):
    """Water level at wave gauges (the paper's experiments record water levels
    at fixed gauges, Sec. 4.4.2): at gauge g, the free-surface particles'
    heights (fs == 1, fluid) averaged with weights w = spline(|r_h| / l) of their
    horizontal distance r_h to the gauge (support 2 l), minus the still-water
    level H.  A gauge with no surface particle within 2 l reads 0.  gauges:
    (G,) x positions in 2-D, (G, 2) x, y positions in 3-D."""
    x = sc.x if x is None else np.asarray(x, dtype=np.float64)
    z = sc.z if z is None else np.asarray(z, dtype=np.float64)
    l, _, _ = radii(sc)
    surf = (np.asarray(fs) == 1) & (sc.type == 0)
    g = np.asarray(gauges, dtype=np.float64).reshape(len(gauges), -1)
    eta = np.zeros(len(g))
    for k in range(len(g)):
        dx = x - g[k, 0]
        r2 = dx * dx
        if sc.dim == 3:
            yy = sc.y if y is None else np.asarray(y, dtype=np.float64)
            dy = yy - g[k, 1]
            r2 = r2 + dy * dy
        w = np.where(surf, _spline(np.sqrt(r2) / l), 0.0)
        den = w.sum()
        eta[k] = (w * z).sum() / den - sc.params["H"] if den > 0 else 0.0
    return eta


def gauge_loss(sc, fs, gauges, x=None, y=None, z=None):
    """Squared water levels summed over the gauges, sum_g eta_g^2."""
    eta = gauge_levels(sc, fs, gauges, x, y, z)
    return float((eta * eta).sum())
