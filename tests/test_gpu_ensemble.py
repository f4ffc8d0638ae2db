"""Batched ensemble (vct_batch_step): scenarios with uneven particle counts and
different bathymetries advanced in one call, side by side (one cooperative
launch for all pressure solves) or one after another, agree with advancing
each on its own."""
import numpy as np
import pytest

from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


def _scenarios():
    rng = np.random.default_rng(2)
    out = []
    for k, (L, d0) in enumerate([(0.6, 0.012), (1.2, 0.01), (0.35, 0.008)]):
        bathy = S.random_bumps(rng, 3, 0.005, 0.02, 0.1 * L, 0.9 * L, 0.05, 0.08, 0.03)
        out.append(S.build_tank(f"ens{k}", 2, "SIGMA", 1.0, bathy,
                                dict(d0=d0, H=0.08, H_hat=0.08, precision=1), L, seed=k))
    return out


def _individual(V, scs, nsteps):
    ref = []
    for sc in scs:
        s = V.Solver(sc)
        st = V.DeviceState(sc)
        s.vct_step(st, nsteps)
        ref.append(st.numpy())
        s.close()
    return ref


def test_batch_serial_equals_individual_steps(monkeypatch):
    """Queued one scenario after another (VCT_BATCH_SERIAL), a batch is exactly
    the individual steps."""
    from paper_2607_28872_b300 import vct as V
    monkeypatch.setenv("VCT_BATCH_SERIAL", "1")
    scs = _scenarios()
    assert len({sc.n for sc in scs}) == 3
    ref = _individual(V, scs, 3)
    solvers = [V.Solver(sc) for sc in scs]
    states = [V.DeviceState(sc) for sc in scs]
    stats = V.vct_batch_step(solvers, states, 3)
    assert len(stats) == 3 and all(s.steps_done == 3 for s in stats)
    for st, r in zip(states, ref):
        g = st.numpy()
        for k in ("x", "z", "u", "w", "p", "jbar"):
            assert np.array_equal(g[k], r[k]), k


def rel(g, o):
    den = np.abs(o).max()
    return np.abs(g - o).max() / den if den > 0 else np.abs(g).max()


@pytest.mark.parametrize("form", ["fly", "explicit"])
def test_batch_concurrent_matches_individual_steps(monkeypatch, form):
    """Side by side (one cooperative launch solves all pressure systems, each
    on its share of the grid), a batch agrees with the individual steps to the
    solver tolerance: the solves stop at the same relative residual (1e-9) with
    partial sums grouped differently, so pressure and velocity agree to the
    mixed-form bound of the parity tests (1e-4), positions to that bound times
    dt |v|, and runs are reproducible bit for bit.  Both solver forms of the
    batch are covered (a batch above 75k particles in total, 30k in 3-D, uses the
    large-system one; VCT_BATCH_FORM forces either)."""
    from paper_2607_28872_b300 import vct as V
    monkeypatch.setenv("VCT_BATCH_FORM", form)
    scs = _scenarios()
    ref = _individual(V, scs, 3)
    out = []
    for rep in range(2):
        solvers = [V.Solver(sc) for sc in scs]
        states = [V.DeviceState(sc) for sc in scs]
        stats = V.vct_batch_step(solvers, states, 3)
        assert all(s.steps_done == 3 for s in stats)
        out.append([st.numpy() for st in states])
    for sc, g, r, g2 in zip(scs, out[0], ref, out[1]):
        f = sc.type == S.FLUID
        for k in ("p", "u", "w"):
            assert rel(g[k][f], r[k][f]) < 1e-4, k
        vmax = np.abs(r["u"][f]).max() + np.abs(r["w"][f]).max() + 1.0
        for k in ("x", "z"):
            assert np.abs(g[k][f] - r[k][f]).max() < 1e-4 * sc.params["dt"] * vmax, k
        for k in ("x", "z", "u", "w", "p", "jbar"):
            assert np.array_equal(g[k], g2[k]), k


def test_batch_with_mixed_solver_forms(monkeypatch):
    """Scenarios whose contexts chose different solver forms still run side by
    side (every solve in the large-system form), agreeing with the individual
    steps to the solver tolerance; forced one after another they agree
    exactly."""
    from paper_2607_28872_b300 import vct as V
    scs = _scenarios()[:2]
    ref = _individual(V, scs[:1], 2)
    monkeypatch.setenv("VCT_MG_FORM", "explicit")
    ref += _individual(V, scs[1:2], 2)

    def batch():
        monkeypatch.setenv("VCT_MG_FORM", "explicit")
        explicit = V.Solver(scs[1])
        monkeypatch.delenv("VCT_MG_FORM")
        solvers = [V.Solver(scs[0]), explicit]
        states = [V.DeviceState(sc) for sc in scs]
        V.vct_batch_step(solvers, states, 2)
        return [st.numpy() for st in states]

    for sc, g, r in zip(scs, batch(), ref):
        f = sc.type == S.FLUID
        for k in ("p", "u", "w"):
            assert rel(g[k][f], r[k][f]) < 1e-4, k
    monkeypatch.setenv("VCT_BATCH_SERIAL", "1")
    for g, r in zip(batch(), ref):
        for k in ("x", "z", "u", "w", "p"):
            assert np.array_equal(g[k], r[k]), k


def test_batch_rejects_shared_context():
    from paper_2607_28872_b300 import vct as V
    sc = _scenarios()[0]
    s = V.Solver(sc)
    a, b = V.DeviceState(sc), V.DeviceState(sc)
    with pytest.raises(V.VCTError) as e:
        V.vct_batch_step([s, s], [a, b], 1)
    assert e.value.status == V.VCT_ERR_ARG


@pytest.mark.parametrize("form", ["fly", "explicit"])
def test_batch_graph_replay_equals_direct_launches(monkeypatch, form):
    """Side-by-side steps replayed from the captured CUDA graph give exactly the
    results of the same steps launched directly, over a call of 4 steps (two
    replays of one capture), one of 3 (a replay of the same graph and a direct
    step, which leaves the state buffers in the other parity) and one of 2 (a
    capture for that parity)."""
    from paper_2607_28872_b300 import vct as V
    monkeypatch.setenv("VCT_BATCH_FORM", form)
    scs = _scenarios()

    def run(graph):
        if graph:
            monkeypatch.delenv("VCT_BATCH_NOGRAPH", raising=False)
        else:
            monkeypatch.setenv("VCT_BATCH_NOGRAPH", "1")
        solvers = [V.Solver(sc) for sc in scs]
        states = [V.DeviceState(sc) for sc in scs]
        out, replayed, launches = [], [], []
        for n in (4, 3, 2):
            stats = V.vct_batch_step(solvers, states, n)
            assert all(s.steps_done == n for s in stats)
            replayed.append([s.graph_steps for s in stats])
            launches.append([s.kernel_launches for s in stats])
            out.append([st.numpy() for st in states])
        for s in solvers:
            s.close()
        return out, replayed, launches

    g, g_replayed, g_launches = run(True)
    d, d_replayed, d_launches = run(False)
    assert g_replayed == [[4] * 3, [2] * 3, [2] * 3]
    assert d_replayed == [[0] * 3] * 3
    assert g_launches == d_launches
    for call_g, call_d in zip(g, d):
        for a, b in zip(call_g, call_d):
            for k in ("x", "z", "u", "w", "p", "jbar"):
                assert np.array_equal(a[k], b[k]), k


def test_batched_stages_exact_before_the_solve():
    """Every stage of a side-by-side step is one launch over all scenarios that
    runs the scenario's own stage code: after one step the smoothed volumes Jbar
    (set before the solve from the map, the sort and the neighbour lists, Eq.
    VCT_bar_a) are bit-identical to the individual steps'."""
    from paper_2607_28872_b300 import vct as V
    scs = _scenarios()
    ref = _individual(V, scs, 1)
    solvers = [V.Solver(sc) for sc in scs]
    states = [V.DeviceState(sc) for sc in scs]
    V.vct_batch_step(solvers, states, 1)
    for st, r in zip(states, ref):
        assert np.array_equal(st.numpy()["jbar"], r["jbar"])


def test_batch_launches_do_not_grow_with_scenarios(monkeypatch):
    """Side by side, a step is a fixed number of launches (one per stage plus
    the batched solve), counted on the first scenario, whatever the number of
    scenarios; the other scenarios count their own load and store only."""
    from paper_2607_28872_b300 import vct as V
    monkeypatch.setenv("VCT_BATCH_NOGRAPH", "1")
    scs = _scenarios()
    per_step = []
    for m in (2, 3):
        solvers = [V.Solver(sc) for sc in scs[:m]]
        states = [V.DeviceState(sc) for sc in scs[:m]]
        a = V.vct_batch_step(solvers, states, 1)
        b = V.vct_batch_step(solvers, states, 3)
        per_step.append((b[0].kernel_launches - a[0].kernel_launches) / 2)
        assert all(s.kernel_launches == 2 for s in b[1:])
    assert per_step[0] == per_step[1] and per_step[0] <= 40, per_step


def test_batch_with_different_options_per_scenario():
    """Scenarios that run different stages (free-slip walls and regularisation,
    the ISPH operator set and regularisation, neither) in one batch: each batched stage runs only for the
    scenarios that need it, and every scenario agrees with its own steps to the
    solver tolerance."""
    from paper_2607_28872_b300 import vct as V
    scs = _scenarios()
    scs[0].params.update(wall_slip=1, **S.REGULARISATION)
    scs[1].params.update(operators=1, **S.REGULARISATION)
    ref = _individual(V, scs, 2)
    solvers = [V.Solver(sc) for sc in scs]
    states = [V.DeviceState(sc) for sc in scs]
    stats = V.vct_batch_step(solvers, states, 2)
    assert all(s.steps_done == 2 for s in stats)
    for sc, st, r in zip(scs, states, ref):
        g = st.numpy()
        f = sc.type == S.FLUID
        for k in ("p", "u", "w"):
            assert rel(g[k][f], r[k][f]) < 1e-4, k


def test_batch_isolates_a_failing_scenario():
    """A scenario whose step fails inside a batch (a singular SPH(2) moment matrix
    off the free surface) stops at its own status word: the call reports
    VCT_ERR_SINGULAR, that scenario's state is left as it was, and the other
    scenarios, whose stages shared every launch with it, are stepped and agree
    with their own steps to the solver tolerance."""
    from paper_2607_28872_b300 import vct as V
    from test_gpu_failures import _cross
    bad = _cross()
    bad.params["precision"] = 1
    good = _scenarios()[:2]
    ref = _individual(V, good, 2)
    scs = [good[0], bad, good[1]]
    solvers = [V.Solver(sc) for sc in scs]
    states = [V.DeviceState(sc) for sc in scs]
    before = states[1].numpy()
    with pytest.raises(V.VCTError) as e:
        V.vct_batch_step(solvers, states, 2)
    assert e.value.status == V.VCT_ERR_SINGULAR
    after = states[1].numpy()
    for k in ("x", "z", "u", "w", "p"):
        assert np.array_equal(before[k], after[k]), k
    for sc, st, r in zip(good, (states[0], states[2]), ref):
        g = st.numpy()
        f = sc.type == S.FLUID
        for k in ("p", "u", "w"):
            assert rel(g[k][f], r[k][f]) < 1e-4, k


def _scenarios_3d(precision):
    rng = np.random.default_rng(5)
    out = []
    for k, (L, W) in enumerate([(0.17, 0.09), (0.21, 0.11), (0.13, 0.09)]):
        bathy = S.random_bumps(rng, 2, 0.003, 0.01, 0.2 * L, 0.8 * L, 0.03, 0.05, 0.02)
        sc = S.small_tank(dim=3, kind="BFE", L=L, W=W, H=0.06, d0=0.01, seed=10 + k, aspect=2.0,
                          bathy=bathy, with_wave=True, precision=precision, **S.REGULARISATION)
        out.append(sc)
    return out


@pytest.mark.parametrize("form", ["fly", "explicit"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batch_3d_matches_individual_steps(monkeypatch, precision, form):
    """3-D BFE scenarios of uneven sizes side by side, in both precisions and both
    solver forms of the batch: each agrees with its own steps to the solver
    tolerance (FP64 over two steps to 1e-7; mixed over one step to 1e-4, as the
    single-scenario parity: by the second mixed step a near-surface particle's
    free-surface flag, decided in FP32 within its tie band, can differ between the
    two runs and the pressure then differs locally by ~1e-4)."""
    from paper_2607_28872_b300 import vct as V
    monkeypatch.setenv("VCT_BATCH_FORM", form)
    scs = _scenarios_3d(precision)
    assert len({sc.n for sc in scs}) == 3
    nsteps = 2 if precision == 0 else 1
    ref = _individual(V, scs, nsteps)
    solvers = [V.Solver(sc) for sc in scs]
    states = [V.DeviceState(sc) for sc in scs]
    stats = V.vct_batch_step(solvers, states, nsteps)
    assert all(s.steps_done == nsteps for s in stats)
    tol = 1e-7 if precision == 0 else 1e-4
    for sc, st, r in zip(scs, states, ref):
        g = st.numpy()
        f = sc.type == S.FLUID
        for k in ("p", "u", "v", "w"):
            assert rel(g[k][f], r[k][f]) < tol, k
        assert np.array_equal(g["jbar"], r["jbar"])
