"""Parity on the workloads at their stated sizes and lengths.

  * still-water tank (BF over a 1:10 slope, jitter 0.1 d0, FP64): 100 steps,
    the GPU state against the oracle's after every 25 steps;
  * 3-D beach (BFE, aspect 4, 2.1 M fluid particles, mixed): one step of the
    full workload on the GPU, checked element by element at >= 1,000 sampled
    fluid particles against the oracle run on the samples' neighbourhoods only
    (every quantity before the pressure solve depends on particles within
    3 r_e, so the oracle's sub-state holds every particle within 4 r_e of a
    sample);
  * ensemble (64 sigma scenarios, log-uniform sizes): three scenarios of
    different sizes stepped together through vct_batch_step, each against the
    oracle's step of that scenario alone.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


def rel(g, o):
    den = np.abs(o).max()
    return np.abs(np.asarray(g) - np.asarray(o)).max() / (den if den > 0 else 1.0)


def report(tag, value, bound):
    print(f"PARITY {tag} err={value:.3e} bound={bound:.1e}")
    return value < bound


def test_still_water_100_steps_fp64():
    """The still-water tank for its full 100 steps in the FP64 form (solver
    tolerances 1e-12 GPU, 1e-13 oracle): the two trajectories stay within the
    FP64 form's solve bound at every checkpoint."""
    from paper_2607_28872_b300 import vct as V
    sc = S.still_water_bf()
    sc.params.update(krylov_rtol=1e-12, krylov_max_iter=20000)
    f = sc.type == S.FLUID
    solver = V.Solver(sc)
    dst = V.DeviceState(sc)
    ost = O.OracleState(sc)
    for k in range(4):
        solver.vct_step(dst, 25)
        ost, info = O.step(sc, ost, nsteps=25, rtol=1e-13)
        assert info["rc"] == 0
        g = dst.numpy()
        vs = max(np.abs(ost.u[f]).max(), np.abs(ost.w[f]).max())
        tag = f"still_water step {25 * (k + 1)}"
        assert report(f"{tag} p", rel(g["p"][f], ost.p[f]), 1e-6)
        assert report(f"{tag} u/|v|", np.abs(g["u"][f] - ost.u[f]).max() / vs, 1e-5)
        assert report(f"{tag} w/|v|", np.abs(g["w"][f] - ost.w[f]).max() / vs, 1e-5)
        assert report(f"{tag} x/d0", np.abs(g["x"][f] - ost.x[f]).max() / sc.params["d0"], 1e-6)
        assert report(f"{tag} z/d0", np.abs(g["z"][f] - ost.z[f]).max() / sc.params["d0"], 1e-6)


def _clusters(sc, xh, centres, half, halo):
    """Sample set: fluid particles within `half` of each centre (projected, per
    axis); sub-state: every particle within half + halo of a centre."""
    X = xh.T
    f = sc.type == S.FLUID
    sample = np.zeros(sc.n, dtype=bool)
    sub = np.zeros(sc.n, dtype=bool)
    for c in centres:
        d = np.abs(X - np.asarray(c)).max(axis=1)
        sample |= f & (d <= half)
        sub |= d <= half + halo
    return sample, sub


def test_beach_full_size_sampled_parity():
    """One mixed step of the full 3-D beach (2.1 M fluid particles) against the
    oracle at sampled particles: six clusters (deep interior, next to the
    bottom, under the free surface, at a side wall, near the shoreline, under
    the wave crest), each ~7^3 particles, checked element by element for
    lambda_min, rho^, nu, v* and the pressure right side; free-surface flags
    identical outside the tie band."""
    import torch
    from paper_2607_28872_b300 import vct as V
    sc = S.beach_bfe_3d()
    assert sc.n_fluid > 2_000_000
    d0 = sc.params["d0"]
    solver = V.Solver(sc)
    st = V.DeviceState(sc)
    out, stats = solver.vct_step_probe(st)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    del st, solver
    torch.cuda.empty_cache()
    xh, _ = O.projected(sc)
    _, re, _ = O.radii(sc)
    a = sc.aspect
    zt = a * 1.0                                   # projected still-water surface (depth 1 m at x = 0)
    depth = lambda x: 1.0 - 0.05 * x               # noqa: E731
    centres = [(6.0, 2.0, 0.5 * a * depth(6.0)), (8.0, 1.0, 3 * d0), (10.0, 3.0, a * depth(10.0) - 2 * d0),
               (5.0, 0.05, 0.4 * a * depth(5.0)), (17.5, 2.0, 0.5 * a * depth(17.5)),
               (3.0, 2.0, a * depth(3.0) - 3 * d0)]
    sample, sub = _clusters(sc, xh, centres, 3.01 * d0, 4.0 * re)
    assert sample.sum() >= 1000, sample.sum()
    idx = np.flatnonzero(sub)
    part = sc.copy()
    for k in ("x", "y", "z", "u", "v", "w", "p", "jbar", "type"):
        setattr(part, k, getattr(sc, k)[idx].copy())
    _, info = O.step(part, probe=True, max_iter=1)      # the pre-solve fields only
    loc = np.searchsorted(idx, np.flatnonzero(sample))
    gi = np.flatnonzero(sample)
    tol, band = 1e-5, 1e-5
    lam = info["lam_min"][loc]
    lo, hi = sc.params["lam_fs_lo"], sc.params["lam_fs_hi"]
    clear = (np.abs(lam - lo) > band) & (np.abs(lam - hi) > band)
    print(f"PARITY beach samples={gi.size} sub-state={idx.size} tied={int((~clear).sum())} "
          f"free-surface={int(info['fs'][loc].sum())} zt={zt}")
    assert np.array_equal(g["fs"][gi][clear], info["fs"][loc][clear])
    assert report("beach lam_min", rel(g["lam_min"][gi], lam), tol)
    assert report("beach rho_hat", rel(g["rho_hat"][gi], info["rho_hat"][loc]), tol)
    assert report("beach nu", rel(g["nu"][gi], info["nu"][loc]), tol)
    for c in range(3):
        assert report(f"beach vstar{c}", rel(g["vstar"][c][gi], info["vstar"][c][loc]), tol)
    same = clear & (g["fs"][gi] == info["fs"][loc])
    # the stabilisation term's FP32 density estimate: tol |b|_max + (gamma/dt^2) 8 2^-24 rho^_i
    gam = sc.params["gamma_over_dt"] * sc.params["dt"]
    extra = (gam / sc.params["dt"] ** 2) * 8.0 * 2.0 ** -24 * info["rho_hat"][loc][same]
    db = np.abs(g["ppe_b"][gi][same] - info["ppe_b"][loc][same])
    bratio = (db / (tol * np.abs(info["ppe_b"][loc][same]).max() + extra)).max()
    assert report("beach ppe_b/bound", bratio, 1.0)


def test_ensemble_scenarios_against_oracle():
    """Three ensemble scenarios of different sizes (the smallest, one near the
    median, one of ~50k fluid particles) stepped together by vct_batch_step
    (mixed form) against the oracle's step of each scenario alone: pressure,
    velocity and position within the mixed form's solve bounds."""
    from paper_2607_28872_b300 import vct as V
    sizes = S.ensemble_sizes()
    order = np.argsort(sizes)
    pick = [order[0], order[len(order) // 2], int(np.argmin(np.abs(np.asarray(sizes) - 50_000)))]
    scen = S.ensemble()
    chosen = [scen[i] for i in pick]
    for sc in chosen:
        sc.params.update(krylov_rtol=1e-10, krylov_max_iter=20000)
    solvers = [V.Solver(sc) for sc in chosen]
    states = [V.DeviceState(sc) for sc in chosen]
    V.vct_batch_step(solvers, states, 1)
    for k, sc in zip(pick, chosen):
        f = sc.type == S.FLUID
        g = states[chosen.index(sc)].numpy()
        ost, info = O.step(sc, probe=True, rtol=1e-13)
        assert info["rc"] == 0
        tag = f"ensemble[{k}] n_fluid={sc.n_fluid}"
        vs = sc.params["dt"] * (np.abs(ost.u[f]).max() + np.abs(ost.w[f]).max() + 1.0)
        assert report(f"{tag} p", rel(g["p"][f], ost.p[f]), 1e-4)
        assert report(f"{tag} u", rel(g["u"][f], ost.u[f]), 1e-4)
        assert report(f"{tag} w", rel(g["w"][f], ost.w[f]), 1e-4)
        assert report(f"{tag} x/dt|v|", np.abs(g["x"][f] - ost.x[f]).max() / vs, 1e-4)
        assert report(f"{tag} z/dt|v|", np.abs(g["z"][f] - ost.z[f]).max() / vs, 1e-4)
