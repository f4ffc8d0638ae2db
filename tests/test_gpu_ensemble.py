"""Batched ensemble (vct_batch_step): scenarios with uneven particle counts and
different bathymetries advanced in one call give exactly the results of
advancing each on its own."""
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


def test_batch_equals_individual_steps():
    from paper_2607_28872_b300 import vct as V
    scs = _scenarios()
    assert len({sc.n for sc in scs}) == 3
    ref = []
    for sc in scs:
        s = V.Solver(sc)
        st = V.DeviceState(sc)
        s.vct_step(st, 3)
        ref.append(st.numpy())
        s.close()
    solvers = [V.Solver(sc) for sc in scs]
    states = [V.DeviceState(sc) for sc in scs]
    stats = V.vct_batch_step(solvers, states, 3)
    assert len(stats) == 3 and all(s.steps_done == 3 for s in stats)
    for st, r in zip(states, ref):
        g = st.numpy()
        for k in ("x", "z", "u", "w", "p", "jbar"):
            assert np.array_equal(g[k], r[k]), k


def test_batch_rejects_shared_context():
    from paper_2607_28872_b300 import vct as V
    sc = _scenarios()[0]
    s = V.Solver(sc)
    a, b = V.DeviceState(sc), V.DeviceState(sc)
    with pytest.raises(V.VCTError) as e:
        V.vct_batch_step([s, s], [a, b], 1)
    assert e.value.status == V.VCT_ERR_ARG
