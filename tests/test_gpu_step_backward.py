"""Reverse of one time step with respect to the velocities
(vct_step_backward_velocity).

With the positions fixed the step is affine in the fluid velocities v^N, so
the gradient of l = v_bar . v' + x_bar . x' + p_bar . p' is exactly the change
of l for a unit change of one velocity component.  The oracle's step
(Sec. 3.3, Eqs. VCT_predictor, VCT_ppe, PNC, VCT_update) gives every component
that way, one oracle step per component, and the GPU gradient is compared with
it element by element; a second check takes directional differences of the
GPU's own forward step.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu

COMP = {2: ("u", "w"), 3: ("u", "v", "w")}
POS = {2: ("x", "z"), 3: ("x", "y", "z")}


def _tank(kind, dim, precision=0, **extra):
    over = dict(smagorinsky=0, krylov_rtol=1e-12, krylov_max_iter=20000, precision=precision)
    over.update(extra)
    if kind in ("E", "BFE"):
        over["aspect"] = 2.0
    if dim == 2:
        return S.small_tank(dim=2, kind=kind, L=0.12, H=0.06, d0=0.01, seed=3, with_wave=True,
                            **over)
    return S.small_tank(dim=3, kind=kind, L=0.08, W=0.06, H=0.06, d0=0.01, seed=4, **over)


def _weights(sc, seed):
    rng = np.random.default_rng(seed)
    d, n = sc.dim, sc.n
    fl = (sc.type == S.FLUID).astype(float)
    return rng.normal(size=(d, n)) * fl, rng.normal(size=(d, n)) * fl, rng.normal(size=n) * fl


def _oracle_loss(sc, vel, vb, xb, pb):
    st = O.OracleState(sc)
    for c, name in enumerate(COMP[sc.dim]):
        getattr(st, name)[:] = vel[c]
    st, info = O.step(sc, state=st)
    assert info["rc"] == 0
    v1 = np.stack([getattr(st, k) for k in COMP[sc.dim]])
    x1 = np.stack([getattr(st, k) for k in POS[sc.dim]])
    return float((vb * v1).sum() + (xb * x1).sum() + (pb * st.p).sum())


def _base_velocity(sc):
    return np.stack([np.asarray(getattr(sc, k), dtype=np.float64) for k in COMP[sc.dim]])


@pytest.mark.parametrize("kind,dim,precision,slip,tol",
                         [("SIGMA", 2, 0, 0, 1e-9), ("BF", 2, 0, 0, 1e-9), ("E", 2, 0, 0, 1e-9),
                          ("BF", 3, 0, 0, 1e-9), ("BFE", 3, 0, 0, 1e-9), ("SIGMA", 2, 1, 0, 1e-5),
                          ("SIGMA", 2, 0, 1, 1e-9), ("BF", 3, 0, 1, 1e-9),
                          ("SIGMA", 2, 0, 2, 1e-9), ("BF", 3, 0, 2, 1e-9)],
                         ids=["sigma-2d", "bf-2d", "e-2d", "bf-3d", "bfe-3d", "sigma-2d-mixed",
                              "sigma-2d-slip", "bf-3d-slip", "sigma-2d-isph", "bf-3d-isph"])
def test_step_backward_velocity_matches_oracle(kind, dim, precision, slip, tol):
    """Every fluid velocity component's gradient against the oracle's exact
    one-sided difference (the loss is affine in the velocities, free-slip wall
    velocities included).  FP64: to the solves' tolerance; mixed: the
    operators' FP32 sums bound it.  slip 2: no-slip walls under the ISPH
    operator set instead."""
    import torch
    from paper_2607_28872_b300 import vct as V
    extra = dict(operators=1) if slip == 2 else dict(wall_slip=slip)
    sc = _tank(kind, dim, precision, **extra)
    vb, xb, pb = _weights(sc, 11)
    s = V.Solver(sc)
    got, st = s.vct_step_backward_velocity(V.DeviceState(sc), torch.tensor(vb), torch.tensor(xb),
                                           torch.tensor(pb))
    got = got.cpu().numpy()
    assert got.shape == (dim, sc.n)
    fl = np.flatnonzero(sc.type == S.FLUID)
    assert np.all(got[:, sc.type != S.FLUID] == 0.0)
    if fl.size > 100:   # a sample of the particles (one oracle step per component)
        fl = np.sort(np.random.default_rng(5).choice(fl, 100, replace=False))
    v0 = _base_velocity(sc)
    l0 = _oracle_loss(sc, v0, vb, xb, pb)
    h = 0.05
    ref = np.zeros((dim, fl.size))
    for c in range(dim):
        for k, i in enumerate(fl):
            vp = v0.copy()
            vp[c, i] += h
            ref[c, k] = (_oracle_loss(sc, vp, vb, xb, pb) - l0) / h
    scale = np.abs(ref).max()
    err = np.abs(got[:, fl] - ref).max() / scale
    print(f"PARITY step backward velocity {kind} {dim}-D precision {precision} slip {slip}: max err "
          f"{err:.2e} of max |grad| {scale:.3e}, transposed solve {st.krylov_iters_total} iterations")
    assert scale > 0.0
    assert err < tol, err


def _sheared(sc):
    """The scenario's velocities plus a smooth flow whose strain rate is nowhere
    near zero on the fluid (the eddy viscosity's |S| has its kink there)."""
    v = _base_velocity(sc)
    x, z = np.asarray(sc.x), np.asarray(sc.z)
    fl = sc.type == S.FLUID
    v[0] += 0.3 * fl * (1.0 + z / 0.06 + 0.5 * np.sin(2 * np.pi * x / 0.12))
    v[-1] += 0.2 * fl * np.cos(2 * np.pi * x / 0.12)
    return v


def _device_state(sc, vel):
    import torch
    from paper_2607_28872_b300 import vct as V
    st = V.DeviceState(sc)
    for c, k in enumerate(COMP[sc.dim]):
        getattr(st, k)[:] = torch.tensor(vel[c], device="cuda")
    return st


@pytest.mark.parametrize("kind,dim,slip,ops", [("SIGMA", 2, 0, 0), ("BF", 2, 1, 0), ("BF", 3, 0, 0),
                                              ("SIGMA", 2, 0, 1)],
                         ids=["sigma-2d", "bf-2d-slip", "bf-3d", "sigma-2d-isph"])
def test_step_backward_velocity_eddy_viscosity_matches_oracle(kind, dim, slip, ops):
    """With the Smagorinsky model the step is not affine in the velocities: the
    GPU gradient at a sheared flow against the oracle's central differences,
    component by component (a sample of 40 particles in 3-D)."""
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = _tank(kind, dim, wall_slip=slip, smagorinsky=1, operators=ops)
    vb, xb, pb = _weights(sc, 21)
    v0 = _sheared(sc)
    s = V.Solver(sc)
    got, _ = s.vct_step_backward_velocity(_device_state(sc, v0), torch.tensor(vb), torch.tensor(xb),
                                          torch.tensor(pb))
    got = got.cpu().numpy()
    fl = np.flatnonzero(sc.type == S.FLUID)
    if dim == 3:
        fl = np.sort(np.random.default_rng(6).choice(fl, 40, replace=False))
    h = 1e-5
    ref = np.zeros((dim, fl.size))
    for c in range(dim):
        for k, i in enumerate(fl):
            vp, vm = v0.copy(), v0.copy()
            vp[c, i] += h
            vm[c, i] -= h
            ref[c, k] = (_oracle_loss(sc, vp, vb, xb, pb) - _oracle_loss(sc, vm, vb, xb, pb)) / (2 * h)
    scale = np.abs(ref).max()
    err = np.abs(got[:, fl] - ref).max() / scale
    # the eddy viscosity's share, for scale: the same gradient with the model off
    s0 = V.Solver(_tank(kind, dim, wall_slip=slip, operators=ops))
    g0, _ = s0.vct_step_backward_velocity(_device_state(sc, v0), torch.tensor(vb), torch.tensor(xb),
                                          torch.tensor(pb))
    share = np.abs(got - g0.cpu().numpy()).max() / scale
    print(f"PARITY step backward velocity, eddy viscosity, {kind} {dim}-D slip {slip} ops {ops}: max err "
          f"{err:.2e} of max |grad| {scale:.3e}; the model's share of the gradient {share:.2e}")
    assert err < 1e-6, err
    assert share > 100 * err


@pytest.mark.parametrize("kind,dim", [("SIGMA", 2), ("BF", 3)])
def test_step_backward_velocity_matches_gpu_forward(kind, dim):
    """<grad, dv> against (l(v + dv) - l(v - dv)) / 2 of the GPU step itself, for
    random directions dv on the fluid particles."""
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = _tank(kind, dim)
    vb, xb, pb = _weights(sc, 12)
    s = V.Solver(sc)
    got, _ = s.vct_step_backward_velocity(V.DeviceState(sc), torch.tensor(vb), torch.tensor(xb),
                                          torch.tensor(pb))
    got = got.cpu().numpy()
    v0 = _base_velocity(sc)
    fl = (sc.type == S.FLUID).astype(float)

    def loss(vel):
        st = V.DeviceState(sc)
        for c, k in enumerate(COMP[dim]):
            getattr(st, k)[:] = torch.tensor(vel[c], device="cuda")
        V.Solver(sc).vct_step(st, 1)
        v1 = np.stack([getattr(st, k).cpu().numpy() for k in COMP[dim]])
        x1 = np.stack([getattr(st, k).cpu().numpy() for k in POS[dim]])
        return float((vb * v1).sum() + (xb * x1).sum() + (pb * st.p.cpu().numpy()).sum())

    rng = np.random.default_rng(13)
    for _ in range(3):
        dv = rng.normal(size=v0.shape) * fl * 0.01
        fd = (loss(v0 + dv) - loss(v0 - dv)) / 2.0
        an = float((got * dv).sum())
        scale = float(np.abs(got * dv).sum())
        print(f"PARITY step backward velocity vs GPU forward {kind} {dim}-D: "
              f"{an:.9e} against {fd:.9e}")
        assert abs(an - fd) <= 1e-7 * scale, (an, fd, scale)


def test_step_function_autograd():
    """The torch.autograd.Function over a step: vel.grad of a loss on (v', x', p')
    equals the entry's gradient and the GPU step's own directional differences;
    the state passed in is left as it was."""
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = _tank("SIGMA", 2, smagorinsky=1)
    v0 = _sheared(sc)
    s = V.Solver(sc)
    state = _device_state(sc, v0)
    before = {k: getattr(state, k).clone() for k in V.DeviceState.FIELDS}
    vb, xb, pb = [torch.tensor(a, device="cuda") for a in _weights(sc, 31)]
    F = V.step_function()

    def loss(vel):
        v1, x1, p1 = F.apply(vel, s, state)
        return (vb * v1).sum() + (xb * x1).sum() + (pb * p1).sum()

    vel = torch.tensor(v0, device="cuda", requires_grad=True)
    loss(vel).backward()
    for k, t in before.items():
        assert torch.equal(getattr(state, k), t), k
    direct, _ = s.vct_step_backward_velocity(_device_state(sc, v0), vb, xb, pb)
    assert torch.allclose(vel.grad, direct, rtol=0, atol=1e-9 * float(direct.abs().max()))
    fl = torch.tensor((sc.type == S.FLUID).astype(float), device="cuda")
    dv = torch.randn(v0.shape, dtype=torch.float64, device="cuda",
                     generator=torch.Generator(device="cuda").manual_seed(3)) * fl * 1e-5
    with torch.no_grad():
        fd = float(loss(vel + dv) - loss(vel - dv)) / 2.0
    an = float((vel.grad * dv).sum())
    print(f"PARITY step function autograd: {an:.9e} against {fd:.9e}")
    assert abs(an - fd) <= 1e-6 * float((vel.grad * dv).abs().sum())


@pytest.mark.parametrize("dim", [2, 3])
def test_gauge_loss_gradient_through_a_step(dim):
    """The adjoint workload's loss after one step, differentiated with respect to
    the step's starting velocities: vct_gauge_loss's position gradient at the
    updated state, fed to the step reverse as x_bar, against central
    differences of oracle.gauge_loss of the oracle's step (free-surface flags
    of the step held; a sample of 40 fluid particles).  2-D sigma tank with a
    wave; 3-D BFE tank with a wave at aspect 2."""
    import torch
    from paper_2607_28872_b300 import vct as V
    if dim == 2:
        sc = _tank("SIGMA", 2)
        gauges = np.array([0.02, 0.045, 0.07, 0.1])
    else:
        sc = S.small_tank(dim=3, kind="BFE", L=0.2, W=0.08, H=0.05, d0=0.01, seed=4, aspect=2.0,
                          with_wave=True, smagorinsky=0, krylov_rtol=1e-12, krylov_max_iter=20000)
        gauges = np.array([[0.04, 0.03], [0.09, 0.05], [0.15, 0.04]])
    _, info = O.step(sc, probe=True)
    fs = info["fs"].astype(np.int32)
    fs_dev = torch.tensor(fs, device="cuda")
    s = V.Solver(sc)
    st0 = V.DeviceState(sc)
    st1 = st0.clone()
    s.vct_step(st1, 1)
    loss, eta, pos_bar = s.vct_gauge_loss(st1, fs_dev, gauges)
    got, _ = s.vct_step_backward_velocity(st0, None, pos_bar, None)
    got = got.cpu().numpy()
    assert np.abs(eta).max() > 1e-3

    def oracle_loss(vel):
        st = O.OracleState(sc)
        for c, name in enumerate(COMP[dim]):
            getattr(st, name)[:] = vel[c]
        st, inf = O.step(sc, state=st)
        assert inf["rc"] == 0
        return O.gauge_loss(sc, fs, gauges, st.x, st.y if dim == 3 else None, st.z)

    v0 = _base_velocity(sc)
    assert abs(loss - oracle_loss(v0)) <= 1e-8 * loss
    fl = np.flatnonzero(sc.type == S.FLUID)
    fl = np.sort(np.random.default_rng(7).choice(fl, 40, replace=False))
    h = 1e-5
    ref = np.zeros((dim, fl.size))
    for c in range(dim):
        for k, i in enumerate(fl):
            vp, vm = v0.copy(), v0.copy()
            vp[c, i] += h
            vm[c, i] -= h
            ref[c, k] = (oracle_loss(vp) - oracle_loss(vm)) / (2 * h)
    scale = np.abs(ref).max()
    err = np.abs(got[:, fl] - ref).max() / scale
    print(f"PARITY gauge loss through a step, {dim}-D, d loss / d v: max err {err:.2e} of max |grad| "
          f"{scale:.3e}")
    assert scale > 0.0
    assert err < 1e-5, err


@pytest.mark.parametrize("kind,dim,smag,precision,tol",
                         [("SIGMA", 2, 0, 0, 1e-6), ("BF", 2, 1, 0, 1e-6), ("BF", 3, 0, 0, 1e-6),
                          ("SIGMA", 2, 1, 1, 1e-4)],
                         ids=["sigma-2d", "bf-2d-eddy", "bf-3d", "sigma-2d-eddy-mixed"])
def test_step_backward_velocity_regularisation_matches_oracle(kind, dim, smag, precision, tol):
    """With the particle regularisation of the paper's runs (optimized shifting
    0.2, dynamic stabilization at 40 % overlap, XSPH 5e-3 on the free surface)
    on a tank with a strong jitter (pairs inside the stabilization distance)
    and a sheared flow: the GPU gradient against the oracle's central
    differences, component by component (a sample of 40 particles in 3-D)."""
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = _tank(kind, dim, precision, smagorinsky=smag, jitter=0.3, **S.REGULARISATION)
    vb, xb, pb = _weights(sc, 41)
    pb[:] = 0.0   # the step's velocities and positions alone, where the regularisation acts
    v0 = _sheared(sc)
    s = V.Solver(sc)
    got, _ = s.vct_step_backward_velocity(_device_state(sc, v0), torch.tensor(vb), torch.tensor(xb),
                                          torch.tensor(pb))
    got = got.cpu().numpy()
    fl = np.flatnonzero(sc.type == S.FLUID)
    if dim == 3:
        fl = np.sort(np.random.default_rng(8).choice(fl, 40, replace=False))
    h = 1e-6
    ref = np.zeros((dim, fl.size))
    for c in range(dim):
        for k, i in enumerate(fl):
            vp, vm = v0.copy(), v0.copy()
            vp[c, i] += h
            vm[c, i] -= h
            ref[c, k] = (_oracle_loss(sc, vp, vb, xb, pb) - _oracle_loss(sc, vm, vb, xb, pb)) / (2 * h)
    scale = np.abs(ref).max()
    err = np.abs(got[:, fl] - ref).max() / scale
    # the regularisation's share, for scale: the gradient with it off
    s0 = V.Solver(_tank(kind, dim, precision, smagorinsky=smag, jitter=0.3))
    g0, _ = s0.vct_step_backward_velocity(_device_state(sc, v0), torch.tensor(vb), torch.tensor(xb),
                                          torch.tensor(pb))
    share = np.abs(got - g0.cpu().numpy()).max() / scale
    print(f"PARITY step backward velocity, regularisation, {kind} {dim}-D eddy {smag} precision "
          f"{precision}: max err {err:.2e} of max |grad| {scale:.3e}; the regularisation's share "
          f"{share:.2e}")
    assert err < tol, err
    assert share > 100 * err


def test_step_backward_velocity_needs_an_output():
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = _tank("SIGMA", 2)
    s = V.Solver(sc)
    st = V.DeviceState(sc).struct()
    rc = s.lib.vct_step_backward_velocity(s.ctx, V.C.byref(st), None, None, None, None, None)
    assert rc == V.VCT_ERR_ARG


@pytest.mark.parametrize("name", ["adjoint_sigma", "solitary_sigma"])
def test_step_backward_velocity_full_size(name):
    """At the workloads' full sizes (the adjoint workload's 53k-particle channel
    with the eddy viscosity; the 2-D wave's 42k particles with the particle
    regularisation too), FP64: the step reverse against central differences of
    the GPU's own step along two random directions."""
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = getattr(S, name)(precision=0, krylov_rtol=1e-12, krylov_max_iter=20000)
    d, n = sc.dim, sc.n
    rng = np.random.default_rng(17)
    fl = (sc.type == S.FLUID).astype(float)
    vb = torch.tensor(rng.normal(size=(d, n)) * fl, device="cuda")
    xb = torch.tensor(rng.normal(size=(d, n)) * fl, device="cuda")
    s = V.Solver(sc)
    st0 = V.DeviceState(sc)
    got, _ = s.vct_step_backward_velocity(st0, vb, xb)
    v0 = st0.velocity()
    flt = torch.tensor(fl, device="cuda")

    def loss(vel):
        st = st0.clone()
        st.set_velocity(vel)
        s.vct_step(st, 1)
        return float((vb * st.velocity()).sum() + (xb * st.position()).sum())

    gen = torch.Generator(device="cuda").manual_seed(5)
    for _ in range(2):
        dv = torch.randn(v0.shape, dtype=torch.float64, device="cuda", generator=gen) * flt * 1e-6
        fd = (loss(v0 + dv) - loss(v0 - dv)) / 2.0
        an = float((got * dv).sum())
        scale = float((got * dv).abs().sum())
        print(f"PARITY step backward velocity full size {name} (n={n}): {an:.9e} against {fd:.9e}")
        assert abs(an - fd) <= 1e-5 * scale, (an, fd, scale)
