"""Thin Python binding of the C ABI in include/vct.h (argument marshalling only).

Every stage of the step runs in the CUDA library libvct.so; PyTorch provides
device memory and streams.  The binding raises if the library is missing:
there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvct.so")

VCT_OK, VCT_ERR_ARG, VCT_ERR_CUDA, VCT_ERR_CAPACITY = 0, 1, 2, 3
VCT_ERR_SINGULAR, VCT_ERR_NONFINITE, VCT_ERR_NOCONV, VCT_ERR_TIMEOUT = 4, 5, 6, 7
MAP = {"E": 0, "BF": 1, "BFE": 2, "SIGMA": 3}
VCT_MAX_GAUSS = 32

EXPORTS = ("vct_init", "vct_set_stream", "vct_reset_history", "vct_build_neighbours",
           "vct_build_neighbours_noalloc",
           "sph2_derivatives", "sph2_derivatives_backward", "sph2_gradient_backward_positions",
           "sph2_d2_backward_positions", "vct_ppe_backward_positions", "vct_rho_backward_positions",
           "vct_map_backward", "vct_map_backward_positions", "vct_gauge_loss", "vct_step",
           "vct_batch_step",
           "vct_step_host", "vct_step_probe", "vct_ppe_adjoint", "vct_step_backward_velocity",
           "vct_set_profiling", "vct_stage_times", "vct_last_error", "vct_strerror", "vct_destroy")

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class vct_bathymetry(C.Structure):
    _fields_ = [("h0", C.c_double), ("slope_x", C.c_double), ("slope_y", C.c_double),
                ("cos_amp", C.c_double), ("cos_len", C.c_double), ("n_gauss", C.c_int32),
                ("reserved", C.c_int32), ("amp", _dp), ("cx", _dp), ("cy", _dp), ("width", _dp)]


class vct_params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("reserved0", C.c_int32)] + [
        (k, C.c_double) for k in ("rho", "nu_k", "g", "dt", "d0", "l_over_d0", "re_over_l",
                                  "gamma_over_dt", "cv_over_dt", "cs", "ds", "H", "H_hat",
                                  "alpha_min", "alpha_max", "lam_fs_lo", "lam_fs_hi",
                                  "krylov_rtol")] + [
        ("krylov_max_iter", C.c_int32), ("smagorinsky", C.c_int32), ("precision", C.c_int32),
        ("volume_mode", C.c_int32), ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
        ("max_neighbours", C.c_int32), ("preconditioner", C.c_int32),
        ("ops_shift", C.c_double), ("ds_overlap", C.c_double), ("xsph_eps", C.c_double),
        ("spin_limit", C.c_int64), ("operators", C.c_int32), ("wall_slip", C.c_int32),
        ("cell_over_re", C.c_double), ("mg_omega", C.c_double), ("mg_kappa", C.c_double),
        ("solve_form", C.c_int32), ("mg_cycle", C.c_int32)]


class vct_state(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in
                                     ("x", "y", "z", "u", "v", "w", "p", "jbar", "type")]


class vct_stats(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("krylov_iters_total", C.c_int64),
                ("krylov_iters_max", C.c_int32), ("graph_steps", C.c_int32),
                ("last_residual", C.c_double), ("ppe_rows", C.c_int64), ("ppe_nnz", C.c_int64),
                ("kernel_launches", C.c_int64), ("solve_form", C.c_int32), ("mg_cycle", C.c_int32)]


STAGES = ("load", "map", "sort", "neighbours", "smoothing", "pass1", "pass2", "rhs", "precond",
          "krylov",
          "corrector", "regularise", "store")


class vct_probe(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("fs", "rho_hat", "nu", "lam_min", "vstar", "ppe_b",
                                          "x_test", "ppe_Ax", "jbar_used", "fs_in", "vwall")]


_lib = None


def load_library(path=LIB_PATH):
    """Load libvct.so (built by paper_2607_28872_b300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "`python -m paper_2607_28872_b300.build`; there is no CPU fallback")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.vct_init.argtypes = [C.POINTER(vp), C.POINTER(vct_bathymetry), C.c_int, C.c_double,
                           C.POINTER(vct_params), C.c_int64, vp]
    L.vct_set_stream.argtypes = [vp, vp]
    L.vct_reset_history.argtypes = [vp]
    L.vct_build_neighbours.argtypes = [vp, C.POINTER(vct_state), vp, vp, C.c_int64,
                                       C.POINTER(C.c_int64)]
    L.vct_build_neighbours_noalloc.argtypes = [C.POINTER(vct_bathymetry), C.c_int, C.c_double,
                                               C.POINTER(vct_params), C.POINTER(vct_state), vp,
                                               vp, C.c_int64, C.POINTER(C.c_int64), vp]
    L.vct_build_neighbours_noalloc.restype = C.c_int
    L.sph2_derivatives.argtypes = [vp, C.POINTER(vct_state), vp, C.c_int32, vp, vp, vp]
    L.sph2_derivatives_backward.argtypes = [vp, C.POINTER(vct_state), C.c_int32, vp, vp, vp, vp]
    L.vct_map_backward.argtypes = [vp, C.POINTER(vct_state), vp, vp, vp, vp, vp, vp,
                                   C.POINTER(C.c_double)]
    L.vct_map_backward_positions.argtypes = [vp, C.POINTER(vct_state), vp, vp, vp, vp, vp, vp, vp]
    L.vct_gauge_loss.argtypes = [vp, C.POINTER(vct_state), vp, C.c_int32, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    L.vct_step.argtypes = [vp, C.POINTER(vct_state), C.c_int32, C.POINTER(vct_stats)]
    L.vct_step_host.argtypes = [vp, C.POINTER(vct_state), C.c_int32, C.POINTER(vct_stats)]
    L.vct_batch_step.argtypes = [C.POINTER(vp), C.POINTER(C.POINTER(vct_state)), C.c_int32,
                                 C.c_int32, C.POINTER(vct_stats)]
    L.vct_batch_step.restype = C.c_int
    L.vct_step_probe.argtypes = [vp, C.POINTER(vct_state), C.POINTER(vct_probe),
                                 C.POINTER(vct_stats)]
    L.vct_ppe_adjoint.argtypes = [vp, vp, vp, C.POINTER(vct_stats)]
    L.vct_step_backward_velocity.argtypes = [vp, C.POINTER(vct_state), vp, vp, vp, vp,
                                             C.POINTER(vct_stats)]
    L.sph2_gradient_backward_positions.argtypes = [vp, C.POINTER(vct_state), vp, C.c_int32, vp, vp]
    L.sph2_d2_backward_positions.argtypes = [vp, C.POINTER(vct_state), vp, vp, vp]
    L.vct_ppe_backward_positions.argtypes = [vp, C.POINTER(vct_state), vp, vp, vp]
    L.vct_rho_backward_positions.argtypes = [vp, C.POINTER(vct_state), vp, vp]
    L.vct_set_profiling.argtypes = [vp, C.c_int32]
    L.vct_stage_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    L.vct_last_error.argtypes = [vp, C.POINTER(C.c_int64)]
    L.vct_strerror.argtypes = [C.c_int]
    L.vct_strerror.restype = C.c_char_p
    L.vct_destroy.argtypes = [vp]
    L.vct_destroy.restype = None
    for name in ("vct_init", "vct_set_stream", "vct_reset_history", "vct_build_neighbours",
                 "sph2_derivatives",
                 "sph2_derivatives_backward", "sph2_gradient_backward_positions",
                 "sph2_d2_backward_positions", "vct_ppe_backward_positions",
                 "vct_rho_backward_positions", "vct_map_backward", "vct_map_backward_positions",
                 "vct_gauge_loss",
                 "vct_step", "vct_step_host", "vct_step_probe", "vct_ppe_adjoint",
                 "vct_step_backward_velocity", "vct_set_profiling",
                 "vct_stage_times", "vct_last_error"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def vct_strerror(status):
    return load_library().vct_strerror(int(status)).decode()


class VCTError(RuntimeError):
    def __init__(self, status, where, particle=-1):
        self.status = status
        self.particle = particle
        super().__init__(f"{where}: {vct_strerror(status)} (status {status}, particle {particle})")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def make_bathymetry(b):
    """vct_bathymetry from a scenarios.Bathymetry; returns (struct, keep-alive)."""
    ng = len(b.amp)
    if ng > VCT_MAX_GAUSS:
        raise ValueError("too many Gaussian bumps")
    arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1) if ng else np.zeros(1))
            for a in (b.amp, b.cx, b.cy, b.width)]
    s = vct_bathymetry(b.h0, b.slope_x, b.slope_y, b.cos_amp, b.cos_len, ng, 0,
                       *[a.ctypes.data_as(_dp) for a in arrs])
    return s, arrs


def make_params(sc, **over):
    p = dict(sc.params)
    p.update(over)
    P = vct_params()
    P.dim = sc.dim
    for k in ("rho", "nu_k", "g", "dt", "d0", "l_over_d0", "re_over_l", "gamma_over_dt",
              "cv_over_dt", "cs", "ds", "H", "H_hat", "alpha_min", "alpha_max", "lam_fs_lo",
              "lam_fs_hi", "krylov_rtol"):
        setattr(P, k, float(p[k]))
    P.krylov_max_iter = int(p["krylov_max_iter"])
    P.smagorinsky = int(p["smagorinsky"])
    P.precision = int(p["precision"])
    P.volume_mode = int(p["volume_mode"])
    for k in range(3):
        P.box_lo[k] = float(sc.box_lo[k])
        P.box_hi[k] = float(sc.box_hi[k])
    P.max_neighbours = int(p.get("max_neighbours", 0))
    P.preconditioner = int(p.get("preconditioner", 1))
    for k in ("ops_shift", "ds_overlap", "xsph_eps"):
        setattr(P, k, float(p.get(k, 0.0)))
    P.spin_limit = int(p.get("spin_limit", 0))
    P.operators = int(p.get("operators", 0))
    P.wall_slip = int(p.get("wall_slip", 0))
    for k in ("cell_over_re", "mg_omega", "mg_kappa"):
        setattr(P, k, float(p.get(k, 0.0)))
    P.solve_form = int(p.get("solve_form", 0))
    P.mg_cycle = int(p.get("mg_cycle", 0))
    return P


class DeviceState:
    """Caller-owned particle state as torch CUDA tensors (caller order)."""

    FIELDS = ("x", "y", "z", "u", "v", "w", "p", "jbar")

    def __init__(self, sc, device="cuda"):
        import torch
        self.n = sc.n
        self.dim = sc.dim
        for k in self.FIELDS:
            setattr(self, k, torch.tensor(np.asarray(getattr(sc, k), dtype=np.float64),
                                          device=device))
        self.type = torch.tensor(np.asarray(sc.type, dtype=np.int32), device=device)

    def struct(self):
        return vct_state(self.n, *[_ptr(getattr(self, k)) for k in self.FIELDS], _ptr(self.type))

    def numpy(self):
        out = {k: getattr(self, k).cpu().numpy() for k in self.FIELDS}
        out["type"] = self.type.cpu().numpy()
        return out

    def clone(self):
        out = DeviceState.__new__(DeviceState)
        out.n, out.dim = self.n, self.dim
        for k in self.FIELDS + ("type",):
            setattr(out, k, getattr(self, k).clone())
        return out

    def _names(self, vel):
        if vel:
            return ("u", "w") if self.dim == 2 else ("u", "v", "w")
        return ("x", "z") if self.dim == 2 else ("x", "y", "z")

    def velocity(self):
        """(dim, n) copy of the velocities (u, [v], w)."""
        import torch
        return torch.stack([getattr(self, k) for k in self._names(True)])

    def position(self):
        """(dim, n) copy of the positions (x, [y], z)."""
        import torch
        return torch.stack([getattr(self, k) for k in self._names(False)])

    def set_velocity(self, vel):
        for c, k in enumerate(self._names(True)):
            getattr(self, k).copy_(vel[c])


class HostState:
    """Host (pinned) copy of a particle state for vct_step_host."""

    FIELDS = DeviceState.FIELDS

    def __init__(self, sc, pin=True):
        import torch
        self.n = sc.n
        for k in self.FIELDS:
            t = torch.tensor(np.asarray(getattr(sc, k), dtype=np.float64))
            setattr(self, k, t.pin_memory() if pin else t)
        t = torch.tensor(np.asarray(sc.type, dtype=np.int32))
        self.type = t.pin_memory() if pin else t

    def struct(self):
        return vct_state(self.n, *[_ptr(getattr(self, k)) for k in self.FIELDS], _ptr(self.type))


class Solver:
    """A vct_ctx for one scenario's map, bathymetry and parameters."""

    def __init__(self, sc, capacity=None, stream=None, **over):
        import torch
        self.lib = load_library()
        self.sc = sc
        self.dim = sc.dim
        self.bathy, self._keep = make_bathymetry(sc.bathy)
        self.params = make_params(sc, **over)
        self.capacity = int(capacity or sc.n)
        self.ctx = C.c_void_p()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        rc = self.lib.vct_init(C.byref(self.ctx), C.byref(self.bathy), MAP[sc.map_kind],
                               float(sc.aspect), C.byref(self.params), self.capacity,
                               C.c_void_p(stream.cuda_stream))
        if rc != VCT_OK:
            raise VCTError(rc, "vct_init")

    def _check(self, rc, where):
        if rc != VCT_OK:
            part = C.c_int64(-1)
            self.lib.vct_last_error(self.ctx, C.byref(part))
            raise VCTError(rc, where, part.value)

    def close(self):
        if self.ctx:
            self.lib.vct_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- entry points -----------------------------------------------------
    def vct_build_neighbours(self, state):
        import torch
        s = state.struct()
        nnz = C.c_int64(0)
        row = torch.zeros(state.n + 1, dtype=torch.int64, device="cuda")
        self._check(self.lib.vct_build_neighbours(self.ctx, C.byref(s), _ptr(row), None, 0,
                                                  C.byref(nnz)), "vct_build_neighbours")
        col = torch.zeros(max(nnz.value, 1), dtype=torch.int32, device="cuda")
        self._check(self.lib.vct_build_neighbours(self.ctx, C.byref(s), _ptr(row), _ptr(col),
                                                  col.numel(), C.byref(nnz)),
                    "vct_build_neighbours")
        return row, col[:nnz.value]

    def sph2_derivatives(self, state, phi):
        """phi: (ncomp, n) float64 CUDA tensor -> grad_hat (ncomp, d, n),
        d2_hat (ncomp, m, n), lap_phys (ncomp, n)."""
        import torch
        phi = phi.contiguous()
        nc = phi.shape[0]
        m = 3 if self.dim == 2 else 6
        g = torch.zeros((nc, self.dim, state.n), dtype=torch.float64, device="cuda")
        d2 = torch.zeros((nc, m, state.n), dtype=torch.float64, device="cuda")
        lap = torch.zeros((nc, state.n), dtype=torch.float64, device="cuda")
        s = state.struct()
        self._check(self.lib.sph2_derivatives(self.ctx, C.byref(s), _ptr(phi), nc, _ptr(g),
                                              _ptr(d2), _ptr(lap)), "sph2_derivatives")
        return g, d2, lap

    def sph2_derivatives_backward(self, state, grad_bar=None, d2_bar=None, lap_bar=None):
        """Adjoint of sph2_derivatives w.r.t. phi: returns phi_bar (ncomp, n)."""
        import torch
        ref = next(t for t in (grad_bar, d2_bar, lap_bar) if t is not None)
        nc = ref.shape[0]
        phib = torch.zeros((nc, state.n), dtype=torch.float64, device="cuda")
        c = lambda t: None if t is None else t.contiguous()
        grad_bar, d2_bar, lap_bar = c(grad_bar), c(d2_bar), c(lap_bar)
        s = state.struct()
        self._check(self.lib.sph2_derivatives_backward(self.ctx, C.byref(s), nc, _ptr(grad_bar),
                                                       _ptr(d2_bar), _ptr(lap_bar), _ptr(phib)),
                    "sph2_derivatives_backward")
        return phib

    def vct_map_backward(self, state, zh_bar=None, J_bar=None, sx_bar=None, sy_bar=None,
                         c0_bar=None, c3_bar=None):
        """theta_bar (numpy, 5 + 4 n_gauss): adjoint of the per-particle metric
        (z^, J, s_x, s_y, c0, c3) pulled back to the bathymetry parameters."""
        ng = len(self.sc.bathy.amp)
        out = (C.c_double * (5 + 4 * ng))()
        s = state.struct()
        c = lambda t: None if t is None else _ptr(t.contiguous())
        self._check(self.lib.vct_map_backward(self.ctx, C.byref(s), c(zh_bar), c(J_bar), c(sx_bar),
                                              c(sy_bar), c(c0_bar), c(c3_bar), out),
                    "vct_map_backward")
        return np.array(out[:])

    def vct_map_backward_positions(self, state, zh_bar=None, J_bar=None, sx_bar=None, sy_bar=None,
                                   c0_bar=None, c3_bar=None):
        """(dim, n) float64 CUDA tensor: adjoint of the per-particle metric
        (z^, J, s_x, s_y, c0, c3) pulled back to the physical positions (x, z in
        2-D; x, y, z in 3-D), the identity parts of x^, y^ excluded."""
        import torch
        out = torch.zeros((self.dim, state.n), dtype=torch.float64, device="cuda")
        s = state.struct()
        c = lambda t: None if t is None else _ptr(t.contiguous())
        self._check(self.lib.vct_map_backward_positions(self.ctx, C.byref(s), c(zh_bar), c(J_bar),
                                                        c(sx_bar), c(sy_bar), c(c0_bar), c(c3_bar),
                                                        C.c_void_p(out.data_ptr())),
                    "vct_map_backward_positions")
        return out

    def vct_gauge_loss(self, state, fs, gauges, grad=True):
        """(loss, eta numpy (G,), pos_bar (dim, n) CUDA tensor or None): the
        squared water levels at the gauges and their gradient with respect to
        the physical positions, for the free-surface flags fs (int32 CUDA
        tensor, caller order)."""
        import torch
        g = np.ascontiguousarray(np.asarray(gauges, dtype=np.float64).reshape(-1))
        ng = g.size if self.dim == 2 else g.size // 2
        loss = C.c_double(0.0)
        eta = (C.c_double * max(ng, 1))()
        out = torch.zeros((self.dim, state.n), dtype=torch.float64, device="cuda") if grad else None
        s = state.struct()
        fs = fs.to(torch.int32).contiguous()
        self._check(self.lib.vct_gauge_loss(self.ctx, C.byref(s), C.c_void_p(fs.data_ptr()), ng,
                                            g.ctypes.data_as(C.POINTER(C.c_double)), C.byref(loss),
                                            eta, None if out is None else C.c_void_p(out.data_ptr())),
                    "vct_gauge_loss")
        return loss.value, np.array(eta[:ng]), out

    def sph2_gradient_backward_positions(self, state, phi, grad_bar):
        """Gradient of sum grad_bar . grad_hat (sph2_derivatives' corrected
        gradient) with respect to the projected positions, (dim, n) float64."""
        import torch
        phi = torch.as_tensor(phi, dtype=torch.float64, device="cuda").reshape(-1, state.n).contiguous()
        grad_bar = torch.as_tensor(grad_bar, dtype=torch.float64, device="cuda").contiguous()
        out = torch.zeros((self.dim, state.n), dtype=torch.float64, device="cuda")
        s = state.struct()
        self._check(self.lib.sph2_gradient_backward_positions(
            self.ctx, C.byref(s), C.c_void_p(phi.data_ptr()), int(phi.shape[0]),
            C.c_void_p(grad_bar.data_ptr()), C.c_void_p(out.data_ptr())),
            "sph2_gradient_backward_positions")
        return out

    def sph2_d2_backward_positions(self, state, phi, d2_bar):
        """Gradient of sum d2_bar . d2_hat (sph2_derivatives' second derivatives
        of one field) with respect to the projected positions, (dim, n) float64."""
        import torch
        phi = torch.as_tensor(phi, dtype=torch.float64, device="cuda").reshape(state.n).contiguous()
        d2_bar = torch.as_tensor(d2_bar, dtype=torch.float64, device="cuda").contiguous()
        out = torch.zeros((self.dim, state.n), dtype=torch.float64, device="cuda")
        s = state.struct()
        self._check(self.lib.sph2_d2_backward_positions(
            self.ctx, C.byref(s), C.c_void_p(phi.data_ptr()), C.c_void_p(d2_bar.data_ptr()),
            C.c_void_p(out.data_ptr())), "sph2_d2_backward_positions")
        return out

    def vct_reset_history(self):
        self._check(self.lib.vct_reset_history(self.ctx), "vct_reset_history")

    def vct_ppe_backward_positions(self, state, x, p_bar):
        """Gradient of p_bar . (A x) (the pressure operator's linear part at the
        state's positions) with respect to the projected positions, (dim, n)."""
        import torch
        x = torch.as_tensor(x, dtype=torch.float64, device="cuda").reshape(state.n).contiguous()
        p_bar = torch.as_tensor(p_bar, dtype=torch.float64, device="cuda").reshape(state.n).contiguous()
        out = torch.zeros((self.dim, state.n), dtype=torch.float64, device="cuda")
        s = state.struct()
        self._check(self.lib.vct_ppe_backward_positions(
            self.ctx, C.byref(s), C.c_void_p(x.data_ptr()), C.c_void_p(p_bar.data_ptr()),
            C.c_void_p(out.data_ptr())), "vct_ppe_backward_positions")
        return out

    def vct_rho_backward_positions(self, state, rho_bar):
        """Gradient of sum rho_bar . rho^ (the density estimate) with respect to
        the projected positions, (dim, n) float64."""
        import torch
        rho_bar = torch.as_tensor(rho_bar, dtype=torch.float64, device="cuda").reshape(state.n).contiguous()
        out = torch.zeros((self.dim, state.n), dtype=torch.float64, device="cuda")
        s = state.struct()
        self._check(self.lib.vct_rho_backward_positions(
            self.ctx, C.byref(s), C.c_void_p(rho_bar.data_ptr()), C.c_void_p(out.data_ptr())),
            "vct_rho_backward_positions")
        return out

    def vct_ppe_adjoint(self, p_bar):
        """b_bar = A^-T p_bar for the pressure system of the last step (caller
        order, float64 CUDA tensors of the state's length); returns (b_bar, stats)."""
        import torch
        p_bar = p_bar.to(device="cuda", dtype=torch.float64).contiguous()
        b_bar = torch.zeros_like(p_bar)
        st = vct_stats()
        self._check(self.lib.vct_ppe_adjoint(self.ctx, C.c_void_p(p_bar.data_ptr()),
                                             C.c_void_p(b_bar.data_ptr()), C.byref(st)),
                    "vct_ppe_adjoint")
        return b_bar, st

    def vct_step_backward_velocity(self, state, v_bar=None, x_bar=None, p_bar=None):
        """Gradient with respect to the state's fluid velocities of
        v_bar . v' + x_bar . x' + p_bar . p' after one step from `state`
        (positions held; the state is not advanced).  v_bar, x_bar: (dim, n),
        p_bar: (n,), caller order, each optional; returns ((dim, n) float64 CUDA
        tensor, stats of the transposed pressure solve)."""
        import torch
        d, n = state.dim, state.n

        def dev(a, shape):
            if a is None:
                return None
            return torch.as_tensor(a).to(device="cuda", dtype=torch.float64).reshape(shape).contiguous()
        vb, xb, pb = dev(v_bar, (d, n)), dev(x_bar, (d, n)), dev(p_bar, (n,))
        out = torch.zeros((d, n), dtype=torch.float64, device="cuda")
        ptr = (lambda t: None if t is None else C.c_void_p(t.data_ptr()))
        s = state.struct()
        st = vct_stats()
        self._check(self.lib.vct_step_backward_velocity(self.ctx, C.byref(s), ptr(vb), ptr(xb),
                                                        ptr(pb), ptr(out), C.byref(st)),
                    "vct_step_backward_velocity")
        return out, st

    def vct_step(self, state, nsteps=1):
        s = state.struct()
        st = vct_stats()
        self._check(self.lib.vct_step(self.ctx, C.byref(s), int(nsteps), C.byref(st)), "vct_step")
        return st

    def vct_step_host(self, hstate, nsteps=1):
        s = hstate.struct()
        st = vct_stats()
        self._check(self.lib.vct_step_host(self.ctx, C.byref(s), int(nsteps), C.byref(st)),
                    "vct_step_host")
        return st

    def vct_set_profiling(self, on=True):
        self._check(self.lib.vct_set_profiling(self.ctx, 1 if on else 0), "vct_set_profiling")

    def vct_stage_times(self):
        """{stage: (device ms, bracketed launches)} accumulated while profiling."""
        ms = (C.c_double * len(STAGES))()
        cnt = (C.c_int64 * len(STAGES))()
        self._check(self.lib.vct_stage_times(self.ctx, ms, cnt), "vct_stage_times")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(STAGES)}

    def vct_step_probe(self, state, x_test=None, fs_in=None):
        """One step that also exports intermediate fields.  fs_in: optional int32
        CUDA tensor of free-surface flags (caller order) to use instead of the
        step's own (parity checks pass the oracle's flags)."""
        import torch
        n, d = state.n, self.dim
        out = dict(fs=torch.zeros(n, dtype=torch.int32, device="cuda"),
                   rho_hat=torch.zeros(n, dtype=torch.float64, device="cuda"),
                   nu=torch.zeros(n, dtype=torch.float64, device="cuda"),
                   lam_min=torch.zeros(n, dtype=torch.float64, device="cuda"),
                   vstar=torch.zeros((d, n), dtype=torch.float64, device="cuda"),
                   ppe_b=torch.zeros(n, dtype=torch.float64, device="cuda"),
                   jbar_used=torch.zeros(n, dtype=torch.float64, device="cuda"),
                   vwall=torch.zeros((d, n), dtype=torch.float64, device="cuda"))
        if x_test is not None:
            out["ppe_Ax"] = torch.zeros(n, dtype=torch.float64, device="cuda")
            x_test = x_test.contiguous()
        if fs_in is not None:
            fs_in = fs_in.to(dtype=torch.int32).contiguous()   # kept alive until the call returns
        pr = vct_probe(_ptr(out["fs"]), _ptr(out["rho_hat"]), _ptr(out["nu"]),
                       _ptr(out["lam_min"]), _ptr(out["vstar"]), _ptr(out["ppe_b"]),
                       _ptr(x_test), _ptr(out.get("ppe_Ax")), _ptr(out["jbar_used"]),
                       _ptr(fs_in), _ptr(out["vwall"]))
        s = state.struct()
        st = vct_stats()
        self._check(self.lib.vct_step_probe(self.ctx, C.byref(s), C.byref(pr), C.byref(st)),
                    "vct_step_probe")
        return out, st


def vct_build_neighbours_noalloc(sc, state, row_ptr, col, stream=None, **over):
    """Neighbour CSR without a context and without any device allocation (for
    callers that cannot allocate device memory).  row_ptr: int64 CUDA tensor of
    n+1 entries; col: int32 CUDA tensor (or None to get only nnz).  Returns
    (status, nnz); the limits are 16384 particles and 32768 cells.  `over`
    overrides scenario parameters (box_lo/box_hi: 3-tuples)."""
    import torch
    lib = load_library()
    bathy, keep = make_bathymetry(sc.bathy)
    box = {k: over.pop(k) for k in ("box_lo", "box_hi") if k in over}
    params = make_params(sc, **over)
    for k, v in box.items():
        for a in range(3):
            getattr(params, k)[a] = float(v[a])
    s = state.struct()
    nnz = C.c_int64(0)
    if stream is None:
        stream = torch.cuda.current_stream()
    rc = lib.vct_build_neighbours_noalloc(C.byref(bathy), MAP[sc.map_kind], float(sc.aspect),
                                          C.byref(params), C.byref(s), _ptr(row_ptr), _ptr(col),
                                          0 if col is None else col.numel(), C.byref(nnz),
                                          C.c_void_p(stream.cuda_stream))
    return rc, nnz.value


def sph2_function():
    """torch.autograd.Function over sph2_derivatives: forward and backward both
    run in the CUDA library (backward = sph2_derivatives_backward)."""
    import torch

    class SPH2Derivatives(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phi, solver, state):
            g, d2, lap = solver.sph2_derivatives(state, phi.detach())
            ctx.solver = solver
            ctx.state = state
            return g, d2, lap

        @staticmethod
        def backward(ctx, gbar, d2bar, lapbar):
            phib = ctx.solver.sph2_derivatives_backward(ctx.state, gbar, d2bar, lapbar)
            return phib, None, None

    return SPH2Derivatives


def step_function():
    """torch.autograd.Function over one time step as a function of the velocities,
    the positions held: apply(vel, solver, state) runs vct_step on a copy of
    `state` with velocities `vel` ((dim, n), caller order) and returns
    (v', x', p'); backward is vct_step_backward_velocity at `vel`.  `state` is
    not modified."""
    import torch

    class StepVelocity(torch.autograd.Function):
        @staticmethod
        def forward(ctx, vel, solver, state):
            vel = vel.detach()
            st = state.clone()
            st.set_velocity(vel)
            solver.vct_step(st, 1)
            ctx.solver = solver
            ctx.state = state
            ctx.save_for_backward(vel)
            return st.velocity(), st.position(), st.p.clone()

        @staticmethod
        def backward(ctx, vbar, xbar, pbar):
            (vel,) = ctx.saved_tensors
            st = ctx.state.clone()
            st.set_velocity(vel)
            g, _ = ctx.solver.vct_step_backward_velocity(st, vbar, xbar, pbar)
            return g, None, None

    return StepVelocity


def vct_batch_step(solvers, states, nsteps=1):
    """Advance several scenarios (one Solver and one DeviceState each) in one
    call; returns the list of per-scenario vct_stats."""
    lib = load_library()
    n = len(solvers)
    ctxs = (C.c_void_p * n)(*[s.ctx.value for s in solvers])
    structs = [st.struct() for st in states]
    # vct_state* const* : an array of pointers to the structs
    arr = (C.POINTER(vct_state) * n)(*[C.pointer(x) for x in structs])
    stats = (vct_stats * n)()
    rc = lib.vct_batch_step(ctxs, arr, n, int(nsteps), stats)
    if rc != VCT_OK:
        raise VCTError(rc, "vct_batch_step")
    return list(stats)


class Checkpointer:
    """Checkpointed forward run for a reverse sweep over steps (the adjoint
    workload keeps a checkpoint every 20 steps): a copy of the state every
    `every` steps, and the states of one segment recomputed from its checkpoint
    on demand.  The context's pressure history is reset at every checkpoint,
    on the forward run and on the replays alike, so a replay reproduces the
    forward run's states bit for bit.  The resets change the pressure solve's
    initial guess, so a checkpointed run agrees with the same steps queued by
    vct_step without resets to the solver tolerance only: a finite-difference
    or oracle gradient must use the same reset schedule as the run it checks."""

    def __init__(self, solver, every=20):
        self.solver = solver
        self.every = int(every)
        self.snapshots, self.lengths = [], []

    @staticmethod
    def _copy(state):
        import copy
        out = copy.copy(state)
        for k in DeviceState.FIELDS + ("type",):
            setattr(out, k, getattr(state, k).clone())
        return out

    def run(self, state, nsteps):
        """Advance `state` by nsteps, keeping a checkpoint at every segment start."""
        self.snapshots, self.lengths = [], []
        done = 0
        while done < nsteps:
            k = min(self.every, nsteps - done)
            self.snapshots.append(self._copy(state))
            self.lengths.append(k)
            self.solver.vct_reset_history()
            self.solver.vct_step(state, k)
            done += k
        return state

    def replay(self, seg):
        """The states after each step of segment `seg`, recomputed from its
        checkpoint (a list of DeviceState copies; the checkpoint is kept)."""
        state = self._copy(self.snapshots[seg])
        self.solver.vct_reset_history()
        out = []
        for _ in range(self.lengths[seg]):
            self.solver.vct_step(state, 1)
            out.append(self._copy(state))
        return out
