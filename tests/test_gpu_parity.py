"""Parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Both sides get the same seeded inputs from the scenario generator and share
no code.  Tolerances:
  * neighbour lists: bit-exact (integer work);
  * FP64 form: 1e-12 normwise relative per field (max|gpu - oracle| / max|oracle|)
    for every quantity computed without the pressure solve;
  * pressure after the solve: both sides stop at a relative residual (GPU
    rtol 1e-12, oracle 1e-13), so |dp|/|p| <= kappa(A) (rtol_gpu + rtol_oracle);
    kappa of these operators is below 1e4 (measured on the oracle's dense
    matrix of the small tanks), giving the 1e-7 bound used here;
  * mixed form: FP32 neighbour sums with compensation on ~20 terms and an
    FP64 solve, 1e-5 normwise relative (the stated default).
Free-surface flags are compared outside a tie band |lambda - threshold| < 1e-9
(FP64) / 1e-5 (mixed), where the decision is a threshold on a rounded value.
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
    g = np.asarray(g, dtype=np.float64)
    o = np.asarray(o, dtype=np.float64)
    den = np.abs(o).max()
    if den == 0:
        return np.abs(g).max()
    return np.abs(g - o).max() / den


SMALL = [
    ("bf2d", lambda: S.small_tank(dim=2, kind="BF", L=0.37, H=0.1, d0=0.01, seed=1,
                                  bathy=S.Bathymetry(h0=-0.02, slope_x=0.1))),
    ("sigma2d", lambda: S.small_tank(dim=2, kind="SIGMA", L=0.41, H=0.1, d0=0.01, seed=2,
                                     with_wave=True)),
    ("e2d", lambda: S.small_tank(dim=2, kind="E", L=0.3, H=0.1, d0=0.01, seed=3, aspect=2.5,
                                 bathy=S.Bathymetry())),
    ("bfe3d", lambda: S.small_tank(dim=3, kind="BFE", L=0.17, W=0.09, H=0.06, d0=0.01, seed=4,
                                   aspect=2.0)),
    ("sigma3d", lambda: S.small_tank(dim=3, kind="SIGMA", L=0.15, W=0.11, H=0.07, d0=0.01,
                                     seed=5)),
]


@pytest.mark.parametrize("name,make", SMALL + [("still_water_bf", S.still_water_bf)],
                         ids=[s[0] for s in SMALL] + ["still_water_bf"])
def test_neighbours_bit_exact(vct, name, make):
    sc = make()
    solver = vct.Solver(sc)
    st = vct.DeviceState(sc)
    row, col = solver.vct_build_neighbours(st)
    xh, _ = O.projected(sc)
    l, re, re2 = O.radii(sc)
    orow, ocol = O.neighbours(sc.dim, xh, re, re2, mode=1)
    assert np.array_equal(row.cpu().numpy(), orow)
    assert np.array_equal(col.cpu().numpy(), ocol)


@pytest.mark.parametrize("dim", [2, 3])
def test_neighbours_bit_exact_at_the_radius(vct, dim):
    """Particle pairs at r_e (1 + delta), delta from -1e-2 to 1e-2 down to 1e-8
    and 0, along x, along a diagonal and (3-D) along a space diagonal, near the
    origin and 5.5 m from it: the search's FP32 first test decides outside its
    error bound, the FP64 predicate within it, and the lists are the oracle's
    FP64 predicate's exactly."""
    d0 = 0.01
    params = dict(S.DEFAULT_PARAMS)
    params.update(d0=d0, H=1.0, H_hat=1.0, dt=1e-3)
    sc0 = S.Scenario(name="radius", dim=dim, map_kind="E", aspect=1.0, bathy=S.Bathymetry(),
                     params=params, x=np.zeros(1), y=np.zeros(1), z=np.zeros(1), u=np.zeros(1),
                     v=np.zeros(1), w=np.zeros(1), p=np.zeros(1), jbar=np.ones(1),
                     type=np.zeros(1, np.int32), box_lo=(-0.1, -0.1, -0.1), box_hi=(10.0, 0.6, 0.6))
    _, re, _ = O.radii(sc0)
    deltas = [-1e-2, -1e-3, -3e-4, -1e-4, -3e-5, -1e-5, -1e-6, -1e-8, 0.0,
              1e-8, 1e-6, 1e-5, 3e-5, 1e-4, 3e-4, 1e-3, 1e-2]
    dirs = [(1.0, 0.0, 0.0), (np.cos(0.7), 0.0, np.sin(0.7))]
    if dim == 3:
        dirs.append(tuple(np.array([1.0, 0.6, 0.8]) / np.linalg.norm([1.0, 0.6, 0.8])))
    pts = []
    for x0 in (0.05, 5.5):
        for q, e in enumerate(dirs):
            for k, dl in enumerate(deltas):
                a = np.array([x0 + 5 * re * k, 0.2 if dim == 3 else 0.0, 0.1 + 0.15 * q])
                pts += [a, a + re * (1.0 + dl) * np.array(e)]
    P = np.array(pts)
    n = len(P)
    sc = S.Scenario(name="radius", dim=dim, map_kind="E", aspect=1.0, bathy=S.Bathymetry(),
                    params=params, x=P[:, 0].copy(), y=P[:, 1].copy() if dim == 3 else np.zeros(n),
                    z=P[:, 2].copy(), u=np.zeros(n), v=np.zeros(n), w=np.zeros(n), p=np.zeros(n),
                    jbar=np.ones(n), type=np.zeros(n, np.int32), box_lo=sc0.box_lo, box_hi=sc0.box_hi)
    solver = vct.Solver(sc)
    row, col = solver.vct_build_neighbours(vct.DeviceState(sc))
    xh, _ = O.projected(sc)
    _, re, re2 = O.radii(sc)
    orow, ocol = O.neighbours(dim, xh, re, re2, mode=0)
    assert np.array_equal(row.cpu().numpy(), orow)
    assert np.array_equal(col.cpu().numpy(), ocol)
    # the cases exist on both sides of the radius
    pair = np.diff(orow)[0::2]
    assert pair.min() == 0 and pair.max() == 1


def test_neighbours_bit_exact_sigma_solitary(vct):
    sc = S.solitary_sigma()
    solver = vct.Solver(sc)
    row, col = solver.vct_build_neighbours(vct.DeviceState(sc))
    xh, _ = O.projected(sc)
    l, re, re2 = O.radii(sc)
    orow, ocol = O.neighbours(2, xh, re, re2, mode=1)
    assert np.array_equal(row.cpu().numpy(), orow)
    assert np.array_equal(col.cpu().numpy(), ocol)


def _fields(sc):
    xh, _ = O.projected(sc)
    rng = np.random.default_rng(17)
    X = xh
    d = sc.dim
    a = rng.normal(size=(3, d))
    phis = [np.sin(3.0 * X[0] + 1.0) * np.cos(2.0 * X[-1]),
            0.3 + a[0] @ X + 0.5 * (X ** 2).sum(axis=0) * a[1, 0],
            np.exp(0.5 * X[0]) * (1 + X[-1] ** 2)]
    return np.stack(phis)


# Second derivatives (and the Laplacian built from them) at FREE-SURFACE particles:
# their support is one-sided, so after the linear part is projected out of q_ij
# (p_ij = q_ij - C~^T r_ij) the moment matrix M_i is much worse conditioned than
# in the interior.  D = 2 M^-1 b then carries the rounding of M and b amplified by
# cond(M_i): |dD_i| <= cond_1(M_i) (|dM|/|M| + |db|/|b|) |D_i|.  Each entry of M
# and b is a sum of n_i pair terms of m-vector products, so its rounding is at most
# ~(n_i + m^2) eps relative to the sum of magnitudes (eps = 2^-53 in the FP64 form;
# in the mixed form the pair inputs are FP32 roundings, eps = 2^-24).  The right
# side b sums phi_ij - r_ij . <grad phi>_i, a difference that cancels the field's
# first-order part: its rounding is relative to |grad phi| |r| ~ |grad phi| d0, not
# to the second derivatives.  The bound at each free-surface particle is therefore
# 4 (n_i + m^2) cond_1(M_i) eps (|D_i| + |grad phi_i| / d0), with cond_1(M_i) from
# the oracle's own M_i, relative to the field's scale.  Every other fluid particle
# is held to the strict bounds.
EPS = {0: 2.0 ** -53, 1: 2.0 ** -24}


def report(tag, value, bound):
    """Print a measured error next to its bound (collected in the GPU logs)."""
    print(f"PARITY {tag} err={value:.3e} bound={bound:.1e}")
    return value < bound


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make", SMALL, ids=[s[0] for s in SMALL])
def test_sph2_derivatives_parity(vct, name, make, precision, tol):
    import torch
    sc = make()
    sc.params["precision"] = precision
    phi = _fields(sc)
    solver = vct.Solver(sc)
    g, d2, lap = solver.sph2_derivatives(vct.DeviceState(sc), torch.tensor(phi, device="cuda"))
    og, od2, olap = O.sph2_derivatives(sc, phi)
    _, info = O.step(sc, probe=True)
    fs = info["fs"] == 1
    f = sc.type == S.FLUID
    M = O.moment_matrices(sc)
    m = M.shape[1]
    xh, _ = O.projected(sc)
    _, re, re2 = O.radii(sc)
    row, col = O.neighbours(sc.dim, xh, re, re2)
    nb = np.diff(row)
    cond = np.zeros(sc.n)
    for i in np.flatnonzero(f & fs):
        cond[i] = np.linalg.cond(M[i], 1)
    fs_bound = 4.0 * (nb + m * m) * cond * EPS[precision]
    d0 = sc.params["d0"]
    g, d2, lap = g.cpu().numpy(), d2.cpu().numpy(), lap.cpu().numpy()
    # normwise per field: a gradient or a second-derivative set is one field
    for c in range(phi.shape[0]):
        assert report(f"{name} p{precision} grad{c}", rel(g[c], og[c]), tol)
        sd = np.abs(od2[c]).max()
        sl = np.abs(olap[c]).max()
        e2 = np.abs(d2[c] - od2[c]).max(axis=0) / sd
        el = np.abs(lap[c] - olap[c]) / sl
        assert report(f"{name} p{precision} d2 interior{c}", e2[f & ~fs].max(), tol)
        assert report(f"{name} p{precision} lap interior{c}", el[f & ~fs].max(), tol)
        if (f & fs).any():
            k = np.flatnonzero(f & fs)
            # the particle's own magnitudes relative to the field's scale
            mag2 = (np.abs(od2[c][:, k]).max(axis=0) + np.abs(og[c][:, k]).max(axis=0) / d0) / sd
            magl = (np.abs(olap[c][k]) + np.abs(og[c][:, k]).max(axis=0) / d0) / sl
            r2 = (e2[k] / np.maximum(fs_bound[k] * mag2, tol)).max()
            rl = (el[k] / np.maximum(fs_bound[k] * magl, tol)).max()
            print(f"PARITY {name} p{precision} free-surface cond max {cond[k].max():.2e} "
                  f"d2 err {e2[k].max():.2e} lap err {el[k].max():.2e}")
            assert report(f"{name} p{precision} d2 fs/bound{c}", r2, 1.0)
            assert report(f"{name} p{precision} lap fs/bound{c}", rl, 1.0)


def _probe_compare(vct, sc, precision, tol, band, name="case"):
    """One step through vct_step_probe against the oracle's probe.

    Free-surface flags must agree outside the tie band.  Inside it both
    decisions are correct roundings of the same threshold test; when they
    differ, the GPU step is repeated with the oracle's flags (the probe's
    fs_in), so the pressure system, the solve and the corrector are compared
    on every case.  Returns (stats, number of tied particles, forced)."""
    import torch
    sc = sc.copy()
    sc.params["precision"] = precision
    sc.params["krylov_rtol"] = 1e-12 if precision == 0 else 1e-10
    sc.params["krylov_max_iter"] = 20000
    n = sc.n
    rng = np.random.default_rng(5)
    xt = rng.normal(size=n)
    xt_d = torch.tensor(xt, device="cuda")
    solver = vct.Solver(sc)
    st = vct.DeviceState(sc)
    out, stats = solver.vct_step_probe(st, xt_d)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    gs = st.numpy()
    ost, info = O.step(sc, probe=True, x_test=xt, rtol=1e-13)
    assert info["rc"] == 0
    f = sc.type == S.FLUID
    lam = info["lam_min"]
    lo, hi = sc.params["lam_fs_lo"], sc.params["lam_fs_hi"]
    # thresholds: free surface lo / hi, isolated 0.05
    clear = f & (np.abs(lam - lo) > band) & (np.abs(lam - hi) > band) & (np.abs(lam - 0.05) > band)
    assert np.array_equal(g["fs"][clear], info["fs"][clear])
    tied = f & ~clear
    if precision == 0:
        assert np.array_equal(g["fs"], info["fs"]), "flags differ"
    tag = f"{name} p{precision}"
    assert report(f"{tag} lam_min", rel(g["lam_min"][f], lam[f]), tol)
    assert report(f"{tag} rho_hat", rel(g["rho_hat"][f], info["rho_hat"][f]), tol)
    assert report(f"{tag} nu", rel(g["nu"][f], info["nu"][f]), tol)
    assert report(f"{tag} jbar", rel(g["jbar_used"], info["jbar_used"]), tol)
    for c in range(sc.dim):
        assert report(f"{tag} vstar{c}", rel(g["vstar"][c][f], info["vstar"][c][f]), tol)
    forced = not np.array_equal(g["fs"], info["fs"])
    if forced:
        solver2 = vct.Solver(sc)
        st2 = vct.DeviceState(sc)
        fs_in = torch.tensor(info["fs"], dtype=torch.int32, device="cuda")
        out, stats = solver2.vct_step_probe(st2, xt_d, fs_in=fs_in)
        g = {k: v.cpu().numpy() for k, v in out.items()}
        gs = st2.numpy()
        assert np.array_equal(g["fs"], info["fs"])
    print(f"PARITY {tag} tied={int(tied.sum())} differing={int((g['fs'] != info['fs']).sum())} "
          f"forced={forced}")
    # identical unknown set: the linear system itself, then the solve and the corrector.
    # The right side's stabilisation term gamma (rho Jbar/J - rho^)/dt^2 takes the
    # difference of the target and the density estimate; in the mixed form rho^ is a
    # compensated FP32 sum, exact to a few 2^-24 rho^, so a row's right side is held
    # to tol |b|_max + (gamma/dt^2) 8 2^-24 rho^_i (the FP64 form: tol |b|_max).
    bscale = np.abs(info["ppe_b"]).max()
    gam = sc.params["gamma_over_dt"] * sc.params["dt"]
    extra = (gam / sc.params["dt"] ** 2) * 8.0 * 2.0 ** -24 * info["rho_hat"] if precision else 0.0
    bratio = (np.abs(g["ppe_b"] - info["ppe_b"]) / (tol * bscale + extra)).max()
    assert report(f"{tag} ppe_b/bound", bratio, 1.0)
    assert report(f"{tag} ppe_Ax", rel(g["ppe_Ax"], info["ppe_Ax"]), tol)
    # The solve: the GPU pressure must solve the ORACLE's FP64 system with normwise
    # backward error eta = |A p - b| / (|A| |p| + |b|) within the form's tolerance
    # (independent of the system's conditioning; |A| estimated from below by
    # |A x| / |x| for the random x above, which only makes eta larger).
    unk = f & (info["fs"] == 0)
    if unk.any():
        _, ip = O.step(sc, probe=True, x_test=np.where(unk, gs["p"], 0.0), max_iter=1)
        res = np.abs(ip["ppe_Ax"][unk] - info["ppe_b"][unk]).max()
        a_norm = np.abs(info["ppe_Ax"][unk]).max() / np.abs(xt[unk]).max()
        eta = res / (a_norm * np.abs(gs["p"][unk]).max() + np.abs(info["ppe_b"][unk]).max())
        assert report(f"{tag} solve backward error", eta, tol)
    # forward errors of the solved fields (both sides stop at a residual; the
    # error is at most cond(A) times the backward error): regression bounds
    ptol = 1e-7 if precision == 0 else 1e-4
    assert report(f"{tag} p", rel(gs["p"][f], ost.p[f]), ptol)
    for k in ("u", "w") + (("v",) if sc.dim == 3 else ()):
        assert report(f"{tag} {k}", rel(gs[k][f], getattr(ost, k)[f]), ptol)
    vs = sc.params["dt"] * (np.abs(ost.u[f]).max() + np.abs(ost.w[f]).max() + 1.0)
    for k in ("x", "z") + (("y",) if sc.dim == 3 else ()):
        assert report(f"{tag} {k}/dt|v|", np.abs(gs[k][f] - getattr(ost, k)[f]).max() / vs, ptol)
    return stats, int(tied.sum()), forced


@pytest.mark.parametrize("name,make", SMALL + [("still_water_bf", S.still_water_bf)],
                         ids=[s[0] for s in SMALL] + ["still_water_bf"])
def test_step_parity_fp64(vct, name, make):
    _probe_compare(vct, make(), 0, 1e-12, 1e-9, name)


@pytest.mark.parametrize("name,make", SMALL + [("still_water_bf", S.still_water_bf)],
                         ids=[s[0] for s in SMALL] + ["still_water_bf"])
def test_step_parity_mixed(vct, name, make):
    _probe_compare(vct, make(), 1, 1e-5, 1e-5, name)


def test_step_parity_sigma_solitary_mixed(vct):
    """Full-size sigma solitary wave over a Gaussian bump (~42.5k fluid), mixed form."""
    _probe_compare(vct, S.solitary_sigma(), 1, 1e-5, 1e-5, "solitary")


# Particle regularisation on (dynamic stabilization, XSPH, shifting; Sec. 4.1):
# a jitter of 0.35 d0 puts pairs inside the stabilization distance 0.6 d0.
REG = [
    ("sigma2d_reg", lambda: S.small_tank(dim=2, kind="SIGMA", L=0.41, H=0.1, d0=0.01, seed=6,
                                         with_wave=True, jitter=0.35, **S.REGULARISATION)),
    ("bfe3d_reg", lambda: S.small_tank(dim=3, kind="BFE", L=0.17, W=0.09, H=0.06, d0=0.01,
                                       seed=7, aspect=2.0, jitter=0.35, **S.REGULARISATION)),
]


@pytest.mark.parametrize("precision,tol,band", [(0, 1e-12, 1e-9), (1, 1e-5, 1e-5)],
                         ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make", REG, ids=[r[0] for r in REG])
def test_step_parity_regularised(vct, name, make, precision, tol, band):
    from scipy.spatial import cKDTree
    sc = make()
    xh, _ = O.projected(sc)
    pts = np.asarray(xh).T if np.asarray(xh).shape[0] == sc.dim else np.asarray(xh)
    dmin, _ = cKDTree(pts).query(pts, k=2)
    assert dmin[:, 1].min() < 0.6 * sc.params["d0"]       # stabilization is exercised
    _probe_compare(vct, sc, precision, tol, band, name)


# The multigrid solver has two forms: V-cycle inputs formed on the fly (systems up
# to 75k particles in 2-D, 30k in 3-D) and kept as vectors with cp.async-staged rows (larger ones).
# VCT_MG_FORM forces the large-system form on the small cases; its cycle is V(0,1) through
# the row-cell operator (mg_cycle 2, the default) or V(1,1) (mg_cycle 1).
@pytest.mark.parametrize("cycle", [1, 2], ids=["V11", "V01-rowcell"])
@pytest.mark.parametrize("precision,tol,band", [(0, 1e-12, 1e-9), (1, 1e-5, 1e-5)],
                         ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,make", [SMALL[1], SMALL[3], ("still_water_bf", S.still_water_bf)],
                         ids=[SMALL[1][0], SMALL[3][0], "still_water_bf"])
def test_step_parity_explicit_form(vct, monkeypatch, name, make, precision, tol, band, cycle):
    monkeypatch.setenv("VCT_MG_FORM", "explicit")
    sc = make()
    sc.params["mg_cycle"] = cycle
    _probe_compare(vct, sc, precision, tol, band, f"{name}-explicit-cycle{cycle}")


def test_step_parity_sigma_solitary_explicit_form(vct, monkeypatch):
    monkeypatch.setenv("VCT_MG_FORM", "explicit")
    _probe_compare(vct, S.solitary_sigma(), 1, 1e-5, 1e-5, "solitary-explicit")


def test_forms_agree_over_steps(vct, monkeypatch):
    """Both solver forms and both cycles of the large-system form solve the same system;
    after 20 mixed steps of the still-water tank their states agree to the solver
    tolerance, and the stats name the form and cycle that ran."""
    out = {}
    for form, cycle, want in (("fly", 0, (1, 0)), ("explicit", 1, (2, 1)), ("explicit", 2, (2, 2))):
        monkeypatch.setenv("VCT_MG_FORM", form)
        sc = S.still_water_bf(precision=1)
        sc.params["mg_cycle"] = cycle
        s = vct.Solver(sc)
        st = vct.DeviceState(sc)
        stats = s.vct_step(st, 20)
        assert (stats.solve_form, stats.mg_cycle) == want
        out[(form, cycle)] = st.numpy()
    f = S.still_water_bf().type == S.FLUID
    ref = out[("fly", 0)]
    for key in (("explicit", 1), ("explicit", 2)):
        assert rel(ref["p"][f], out[key]["p"][f]) < 1e-5, key
        assert rel(ref["w"][f], out[key]["w"][f]) < 1e-4, key


def test_multi_step_fp64_matches_oracle(vct):
    sc = S.still_water_bf()
    sc.params.update(krylov_rtol=1e-12, krylov_max_iter=20000)
    solver = vct.Solver(sc)
    st = vct.DeviceState(sc)
    solver.vct_step(st, 5)
    g = st.numpy()
    ost, info = O.step(sc, nsteps=5, rtol=1e-13)
    f = sc.type == S.FLUID
    assert rel(g["p"][f], ost.p[f]) < 1e-6
    assert rel(g["w"][f], ost.w[f]) < 1e-6
    assert np.abs(g["z"][f] - ost.z[f]).max() < 1e-12


def test_host_entry_matches_device(vct):
    sc = S.small_tank(dim=2, kind="SIGMA", L=0.3, H=0.1, d0=0.01, seed=8, with_wave=True)
    s1 = vct.Solver(sc)
    dev = vct.DeviceState(sc)
    s1.vct_step(dev, 3)
    s2 = vct.Solver(sc)
    host = vct.HostState(sc)
    s2.vct_step_host(host, 3)
    g = dev.numpy()
    for k in ("x", "z", "u", "w", "p", "jbar"):
        assert np.array_equal(g[k], getattr(host, k).numpy()), k


def test_run_to_run_bit_identical(vct):
    sc = S.small_tank(dim=2, kind="BF", L=0.3, H=0.1, d0=0.01, seed=9, precision=1)
    outs = []
    for _ in range(2):
        s = vct.Solver(sc)
        st = vct.DeviceState(sc)
        s.vct_step(st, 4)
        outs.append(st.numpy())
    for k in ("x", "z", "u", "w", "p"):
        assert np.array_equal(outs[0][k], outs[1][k]), k


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_graph_steps_equal_direct_steps(vct, monkeypatch, precision):
    """vct_step replays its steps from captured CUDA graphs (one per buffer
    parity); the results are those of the same steps launched directly, bit for
    bit, over calls of 3 steps and then 2 (the second call starts from the other
    parity), and the stats count the replayed steps and the same launches."""
    sc = S.small_tank(dim=2, kind="SIGMA", L=0.3, H=0.1, d0=0.01, seed=8, with_wave=True,
                      precision=precision)

    def run(graph):
        if graph:
            monkeypatch.delenv("VCT_STEP_NOGRAPH", raising=False)
        else:
            monkeypatch.setenv("VCT_STEP_NOGRAPH", "1")
        s = vct.Solver(sc)
        st = vct.DeviceState(sc)
        a = s.vct_step(st, 3)
        b = s.vct_step(st, 2)
        return st.numpy(), (a.graph_steps, b.graph_steps), (a.kernel_launches, b.kernel_launches)

    g, g_steps, g_launches = run(True)
    d, d_steps, d_launches = run(False)
    assert g_steps == (3, 2) and d_steps == (0, 0)
    assert g_launches == d_launches
    for k in ("x", "z", "u", "w", "p", "jbar"):
        assert np.array_equal(g[k], d[k]), k


def test_errors_are_reported(vct):
    sc = S.small_tank(dim=2, kind="BF", L=0.2, H=0.08, d0=0.01, seed=1)
    s = vct.Solver(sc, max_neighbours=8)
    st = vct.DeviceState(sc)
    with pytest.raises(vct.VCTError) as e:
        s.vct_step(st, 1)
    assert e.value.status == vct.VCT_ERR_CAPACITY
    before = st.numpy()
    s2 = vct.Solver(sc, krylov_max_iter=1, krylov_rtol=1e-14)
    st2 = vct.DeviceState(sc)
    with pytest.raises(vct.VCTError) as e:
        s2.vct_step(st2, 1)
    assert e.value.status == vct.VCT_ERR_NOCONV
    after = st2.numpy()
    for k in ("x", "z", "p"):   # failed call leaves the caller's state untouched
        assert np.array_equal(before[k], after[k])
    s3 = vct.Solver(sc, capacity=sc.n)
    big = vct.DeviceState(S.small_tank(dim=2, kind="BF", L=0.3, H=0.08, d0=0.01))
    with pytest.raises(vct.VCTError) as e:
        s3.vct_step(big, 1)
    assert e.value.status == vct.VCT_ERR_CAPACITY


def test_degenerate_inputs(vct):
    """An empty state is an argument error; a state without fluid particles
    steps (nothing moves, no pressure unknowns, no iterations); a batch of one
    scenario is vct_step of that scenario bit for bit."""
    sc = S.small_tank(dim=2, kind="BF", L=0.2, H=0.08, d0=0.01, seed=1)
    s = vct.Solver(sc)
    empty = vct.DeviceState(sc)
    empty.n = 0
    with pytest.raises(vct.VCTError) as e:
        s.vct_step(empty, 1)
    assert e.value.status == vct.VCT_ERR_ARG
    walls = sc.copy()
    walls.type[:] = S.WALL
    s2 = vct.Solver(walls)
    st = vct.DeviceState(walls)
    stats = s2.vct_step(st, 2)
    assert stats.steps_done == 2 and stats.ppe_rows == 0 and stats.krylov_iters_total == 0
    g = st.numpy()
    for k in ("x", "z", "u", "w"):
        assert np.array_equal(g[k], getattr(walls, k)), k
    one = vct.DeviceState(sc)
    vct.vct_batch_step([vct.Solver(sc)], [one], 3)
    ref = vct.DeviceState(sc)
    vct.Solver(sc).vct_step(ref, 3)
    a, b = one.numpy(), ref.numpy()
    for k in ("x", "z", "u", "w", "p", "jbar"):
        assert np.array_equal(a[k], b[k]), k


def test_poisoned_input_nonfinite(vct):
    sc = S.small_tank(dim=2, kind="BF", L=0.2, H=0.08, d0=0.01, seed=1)
    sc.u[3] = np.nan
    s = vct.Solver(sc)
    st = vct.DeviceState(sc)
    with pytest.raises(vct.VCTError) as e:
        s.vct_step(st, 1)
    assert e.value.status in (vct.VCT_ERR_NONFINITE, vct.VCT_ERR_NOCONV)


def test_multi_step_3d_trajectory_matches_oracle(monkeypatch):
    """Ten steps of a 1 m x 0.3 m slice of the 3-D BFE beach (aspect 4, ~36k
    particles): the GPU (FP64 and mixed) follows the oracle's maximum speed step
    by step (the configuration develops the slow growth of the method without
    particle regularisation, which both sides reproduce)."""
    sc0 = S.beach_bfe_3d(L=1.0, W=0.3, x0=0.5)
    f = sc0.type == S.FLUID
    st = O.OracleState(sc0)
    ref = []
    for _ in range(10):
        st, info = O.step(sc0, st, nsteps=1, rtol=1e-9)
        assert info["rc"] == 0
        ref.append(np.sqrt(st.u ** 2 + st.v ** 2 + st.w ** 2)[f].max())
    from paper_2607_28872_b300 import vct as V
    for prec, form in ((0, "fly"), (1, "fly"), (1, "explicit")):
        monkeypatch.setenv("VCT_MG_FORM", form)
        sc = sc0.copy()
        sc.params["precision"] = prec
        s = V.Solver(sc)
        dst = V.DeviceState(sc)
        for k in range(10):
            s.vct_step(dst, 1)
            g = dst.numpy()
            vmax = np.sqrt(g["u"] ** 2 + g["v"] ** 2 + g["w"] ** 2)[f].max()
            assert abs(vmax - ref[k]) <= 2e-3 * ref[k], (prec, form, k, vmax, ref[k])


def test_initial_guess_history(vct, monkeypatch):
    """The solve starts from the pressure extrapolated over the context's last
    steps only when the caller continues the run.  Over 8 steps (in calls of
    one step) the extrapolated and the plain starts agree to the solver
    tolerance; a state the context did not produce (here a fresh copy of the
    scenario) is stepped exactly as by a fresh context."""
    sc = S.solitary_sigma(L=2.0, bump_x=1.0, x0=0.4, precision=1)
    f = sc.type == S.FLUID
    out = {}
    for g in ("0", "2"):
        monkeypatch.setenv("VCT_PGUESS", g)
        s = vct.Solver(sc)
        st = vct.DeviceState(sc)
        for _ in range(8):
            s.vct_step(st, 1)
        out[g] = st.numpy()
        if g == "2":
            used = s
    assert rel(out["2"]["p"][f], out["0"]["p"][f]) < 1e-4
    assert rel(out["2"]["u"][f], out["0"]["u"][f]) < 1e-4
    fresh_state = vct.DeviceState(sc)
    used.vct_step(fresh_state, 1)
    s2 = vct.Solver(sc)
    ref = vct.DeviceState(sc)
    s2.vct_step(ref, 1)
    a, b = fresh_state.numpy(), ref.numpy()
    for k in ("x", "z", "u", "w", "p"):
        assert np.array_equal(a[k], b[k]), k
