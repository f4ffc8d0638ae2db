"""The schedule autotuner's host logic (paper_2607_28872_b300/autotune.py),
with a stand-in timer: one representative per size class, the fastest
successful candidate kept, failed candidates skipped, classes without any
success left out, nearest-class lookup, JSON round trip."""
import json

from paper_2607_28872_b300 import autotune as A
from paper_2607_28872_b300 import scenarios as S


def _scen(n):
    class Sc:
        dim = 2
        params = {"precision": 1}
    s = Sc()
    s.n = n
    return s


def test_tuner_keeps_the_fastest_successful_candidate(tmp_path):
    scs = [_scen(n) for n in (5000, 5200, 5100, 40000, 41000, 160000)]
    seen = []

    def timer(sc, knobs):
        seen.append((sc.n, knobs["cell_over_re"], knobs["mg_omega"], knobs["mg_kappa"]))
        if sc.n == 160000:
            return None                                   # every candidate fails there
        if knobs["mg_kappa"] == 1.5:
            return None                                   # this knob fails everywhere
        # fastest: the larger cells for small systems, omega 0.85 everywhere
        t = 1.0 + abs(knobs["mg_omega"] - 0.85) * 10 + (0.0 if knobs["cell_over_re"] > 1 else 0.5)
        return t + (0.2 if sc.n > 10000 and knobs["cell_over_re"] > 1 else 0.0), 12.0

    table = A.tune(scs, form=2, timer=timer)
    # the representatives are the median-sized members of each class
    reps = {n for n, *_ in seen}
    assert reps == {5100, 41000, 160000}
    assert set(table) == {"d2_p1_n2^12", "d2_p1_n2^15"}       # the 2^17 class failed
    small = table["d2_p1_n2^12"]["knobs"]
    assert small["mg_omega"] == 0.85 and small["mg_kappa"] != 1.5 and small["solve_form"] == 2
    assert all(t["ms_per_step"] is None for t in table["d2_p1_n2^12"]["tried"]
               if t["knobs"]["mg_kappa"] == 1.5)
    path = tmp_path / "t.json"
    A.save(table, path)
    again = A.load(path)
    assert json.loads(json.dumps(table)) == again
    # lookup: own class, nearest class, other dimension -> nothing
    assert A.tuned(_scen(5000), again) == {k: small[k] for k in A.KNOBS}
    assert A.tuned(_scen(300000), again) == {k: again["d2_p1_n2^15"]["knobs"][k] for k in A.KNOBS}
    three = _scen(5000)
    three.dim = 3
    assert A.tuned(three, again) == {}


def test_size_class_of_the_ensemble():
    classes = {A.size_class(sc) for sc in S.ensemble(n_scen=8)}
    assert all(c[0] == 2 and c[1] == 1 for c in classes)
    assert 2 <= len(classes) <= 8
