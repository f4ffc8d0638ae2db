"""Autotuner of the step's schedule, per scenario size class.

An ensemble holds scenarios of very different sizes (5k to 200k particles);
which schedule runs a step fastest depends on the size.  The knobs are the
`vct_params` schedule fields, which change how a step runs but not what it
computes:

  cell_over_re  edge of the background cells over r_e (the neighbour search
                visits the 3^dim adjacent cells; the multigrid's first coarse
                level is the cells, so larger cells also mean coarser
                aggregates);
  mg_omega      Jacobi damping of the multigrid smoother;
  mg_kappa      scale of the coarse-grid correction;
  solve_form    1: small-system form, 2: large-system form of the solver;
  mg_cycle      the large-system form's cycle, 1: V(1,1) through the
                assembled rows, 2: V(0,1) through the row-cell operator.

`tune` times every candidate on one representative scenario per size class
(CUDA events around a few steps after a warm-up, the iterations per step
recorded), drops candidates whose steps fail, keeps the fastest and returns a
table; `save`/`load` store it as JSON; `tuned` gives a scenario the knobs of
its size class (the nearest class when its own was not tuned).  Timing runs
on the GPU through the C ABI; the selection logic is plain Python and is
tested with a stand-in timer.
"""
from __future__ import annotations

import itertools
import json
import math

KNOBS = ("cell_over_re", "mg_omega", "mg_kappa", "solve_form", "mg_cycle")


def candidates(dim, form=0, cycles=(0,)):
    """The schedule grid searched per size class (cycles: the mg_cycle values)."""
    cells = (1.0, 1.25)
    omegas = (0.85, 0.9, 0.95) if dim == 2 else (0.65, 0.7, 0.75)
    kappas = (1.2, 1.3, 1.4, 1.5) if dim == 2 else (1.1, 1.2, 1.3)
    return [dict(cell_over_re=c, mg_omega=w, mg_kappa=k, solve_form=form, mg_cycle=y)
            for c, w, k, y in itertools.product(cells, omegas, kappas, cycles)]


def size_class(sc):
    """(dim, precision, round(log2 of the particle count)) of a scenario."""
    return (int(sc.dim), int(sc.params.get("precision", 0)), int(round(math.log2(max(sc.n, 1)))))


def _key(cls):
    return "d%d_p%d_n2^%d" % cls


def _unkey(key):
    d, p, n = key.split("_")
    return int(d[1:]), int(p[1:]), int(n.split("^")[1])


def time_candidate(sc, knobs, steps=6, warmup=2):
    """Milliseconds per step and Krylov iterations per step of `sc` run with the
    knobs (a fresh context and state), or None if a step fails."""
    import torch

    from . import vct
    try:
        solver = vct.Solver(sc, **knobs)
        state = vct.DeviceState(sc)
        solver.vct_step(state, warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st = solver.vct_step(state, steps)
        e1.record()
        e1.synchronize()
        solver.close()
        return e0.elapsed_time(e1) / steps, st.krylov_iters_total / steps
    except vct.VCTError:
        return None


def tune(scenarios, form=0, timer=time_candidate, grid=candidates):
    """One representative scenario per size class (the median-sized one), every
    candidate of the grid timed on it; returns {class key: entry} with the
    fastest candidate's knobs, its time and every candidate's result."""
    classes = {}
    for sc in scenarios:
        classes.setdefault(size_class(sc), []).append(sc)
    table = {}
    for cls, members in sorted(classes.items()):
        members = sorted(members, key=lambda s: s.n)
        rep = members[len(members) // 2]
        tried = []
        for knobs in grid(cls[0], form):
            r = timer(rep, knobs)
            tried.append(dict(knobs=knobs, ms_per_step=None if r is None else r[0],
                              iters_per_step=None if r is None else r[1]))
        ok = [t for t in tried if t["ms_per_step"] is not None]
        if not ok:
            continue
        best = min(ok, key=lambda t: t["ms_per_step"])
        table[_key(cls)] = dict(knobs=best["knobs"], ms_per_step=best["ms_per_step"],
                                iters_per_step=best["iters_per_step"], n_particles=rep.n,
                                tried=tried)
    return table


def save(table, path):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load(path):
    with open(path) as f:
        return json.load(f)


def tuned(sc, table):
    """The knobs of the scenario's size class: its own class, else the nearest
    tuned class of the same dimension and precision; {} without one."""
    d, p, n = size_class(sc)
    best, dist = None, None
    for key, entry in table.items():
        kd, kp, kn = _unkey(key)
        if (kd, kp) != (d, p):
            continue
        if dist is None or abs(kn - n) < dist:
            best, dist = entry, abs(kn - n)
    return {} if best is None else {k: best["knobs"][k] for k in KNOBS if k in best["knobs"]}
