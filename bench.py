#!/usr/bin/env python3
"""Benchmark of the VCT + SPH(2) step: particle-updates/s per SPH(2) step.

Default workload: the 3-D BFE-SPH solitary wave (H = 0.1 m) on a 1:20 beach,
20 x 4 m basin, depth 1 m shoaling to 0, ellipsoidal particles of aspect
ratio 4, d0 = 0.043 m: 2,105,788 fluid particles (2.59 M with walls), mixed
precision (FP32 compensated neighbour sums, FP64 moment solves and pressure
iterate).  Inputs are the seeded synthetic scenario of
paper_2607_28872_b300.scenarios, resident in HBM before timing.

One step = one call of vct_step for one time step: map + cell sort,
neighbours, SPH(2) passes, predictor, pressure equation, multigrid BiCGSTAB,
corrector, particle regularisation.  The working set (~10 GB) is far above
L2; L2 is also flushed (256 MB write) before every timed step, outside the
timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload beach_bfe_3d|sigma_solitary|...]

--impl reference times the FP64 CPU oracle (the plain reference program of
this project) on the host cores, on a bounded slice of the same workload.
Multi-GPU: independent replicas (the step has no data-parallel split that
avoids per-iteration halo exchange), one per rank, scaling "weak".
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-updates/s per SPH(2) step"
UNIT = "particle-updates/s"
WORKLOAD_2D = ("2-D sigma-SPH solitary wave (H/d=0.2) over a 0.3 m Gaussian bump, 10 m x 0.5 m "
               "channel, d0=1/90 m, mixed FP32/FP64")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="host-buffer steps timed for e2e (default: min(steps, 20))")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--workload", default="beach_bfe_3d", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64-probe", action="store_true",
                    help="skip the per-field error of the mixed form against the FP64 form")
    ap.add_argument("--ensemble-size", type=int, default=64)
    ap.add_argument("--tune", default=None, metavar="PATH",
                    help="ensemble: run the schedule autotuner first and write its table to PATH")
    ap.add_argument("--no-tuning", action="store_true",
                    help="ensemble: run with the built-in schedule, not the tuned table")
    ap.add_argument("--horizon", type=int, default=None,
                    help="restart from the initial state every this many steps (default 150 "
                         "in 2-D, 15 in 3-D; 0 = never)")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="host seconds the reference arm's timed and warm-up steps aim at")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_ms(local_ms, world, device="cuda"):
    """The job's time: the slowest rank's (max over ranks), returned on every
    rank; one replica per GPU, so this reduction is the only exchange."""
    if world <= 1:
        return local_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(units_per_rank, world, steps, ms):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank * steps / (ms / 1e3)


WORKLOADS = {
    "sigma_solitary": WORKLOAD_2D,
    "still_water_bf": "2-D BF still water over a 1:10 slope, 1 m x 0.2 m, d0=0.01 m, jitter 0.1 d0",
    "beach_bfe_3d": ("3-D BFE-SPH solitary wave (H=0.1 m) on a 1:20 beach, 20 x 4 m basin, depth 1 m -> 0, "
                     "aspect ratio 4, d0=0.043 m, mixed FP32/FP64"),
    "beach_bfe_3d_slice": ("3-D BFE solitary wave, 8 x 1.6 m slice of the 1:20 beach (depth 1 -> 0.6 m), "
                           "aspect 4, d0=0.043 m (profiling size)"),
    "ensemble": "sigma-SPH ensemble, particle counts log-uniform 5e3-2e5 (seed 2), 4 bumps each",
    "dam_break_3d": ("3-D sigma-SPH dam break, bottom 0.1 x + 0.02 cos(2 pi x / 0.2) m, projected basin "
                     "25 x 20 x 10 cm, H = 15 cm, H^ = 10 cm, d0 = 0.25 cm, dt = 1e-4 s, column x < 8 cm"),
    "efficiency": ("hydrostatic 1 m tank, H = 0.2 m, bottom 0.12 x + 0.01 (1 - cos(2 pi x / 0.5)): "
                   "BF d0 = 0.2 cm, BFE d0 = 0.5 cm alpha 2.5, sigma d0 = 0.5 cm alpha 1-2.5"),
    "adjoint": ("2-D sigma channel 10 m, flat 0.5 m + 16 random Gaussian bumps (seed 1), d0=0.01 m, "
                "the step's reverse and the operator adjoints"),
}


# DRAM bytes (read + write) of the dominant kernel from one ncu capture of its
# CURRENT version in the mixed form (summaries under profiles/); a workload
# without an entry reports traffic null.  "per_unit": bytes per fluid particle
# per Krylov iteration (the 3-D beach is captured on its 8 x 1.6 m slice; its
# traffic grows with rows x iterations); "per_launch": bytes per launch.
NCU_TRAFFIC = {
    "beach_bfe_3d": ("per_unit", 1690.0, "profiles/k_krylov_mg_beach_bfe_3d_slice_540k.md"),
    "beach_bfe_3d_slice": ("per_unit", 1690.0, "profiles/k_krylov_mg_beach_bfe_3d_slice_540k.md"),
}


def workload(precision=1, name="sigma_solitary"):
    from paper_2607_28872_b300 import scenarios as S
    if name == "still_water_bf":
        return S.still_water_bf(precision=precision)
    if name == "beach_bfe_3d":
        return S.beach_bfe_3d(precision=precision)
    if name == "beach_bfe_3d_slice":
        return S.beach_bfe_3d(L=8.0, W=1.6, precision=precision)
    if name == "dam_break_3d":
        return S.dam_break_sigma_3d(precision=precision)
    return S.solitary_sigma(precision=precision)


def run_adjoint(args):
    """Adjoint/forward times on the 2-D adjoint workload (sigma channel, flat
    0.5 m + 16 random bumps, ~53k fluid).  The line's value is the reverse of one
    whole step with respect to the velocities (vct_step_backward_velocity, which
    re-assembles the step's operators) against one forward step.  Beside it:
    the SPH(2) derivative operator (sph2_derivatives against
    sph2_derivatives_backward, three fields), the pressure solve against its
    transposed solve, and the gauge loss after one step with and without its
    gradient with respect to the starting velocities.  Not the headline line."""
    import numpy as np
    import torch
    from paper_2607_28872_b300 import scenarios as S
    from paper_2607_28872_b300 import vct
    if dist_env()[0] != 0:   # one line per job: rank 0's (replicas only)
        return
    sc = S.adjoint_sigma(precision=args.precision)
    solver = vct.Solver(sc)
    state = vct.DeviceState(sc)
    g = torch.Generator(device="cuda").manual_seed(0)
    phi = torch.randn((3, sc.n), dtype=torch.float64, device="cuda", generator=g)
    gb, db, lb = solver.sph2_derivatives(state, phi)
    gb, db, lb = torch.randn_like(gb), torch.randn_like(db), torch.randn_like(lb)

    def timed(fn, k):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    k = min(args.steps, 50)
    fwd = timed(lambda: solver.sph2_derivatives(state, phi), k)
    bwd = timed(lambda: solver.sph2_derivatives_backward(state, gb, db, lb), k)
    # the pressure solve and its adjoint (transpose solve) on one step of the workload
    solver.vct_set_profiling(True)
    solver.vct_step(state, 1)
    fwd_solve_ms = solver.vct_stage_times()["krylov"][0]
    solver.vct_set_profiling(False)
    pb = torch.randn(sc.n, dtype=torch.float64, device="cuda", generator=g)
    solver.vct_ppe_adjoint(pb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, ast = solver.vct_ppe_adjoint(pb)
    e1.record()
    e1.synchronize()
    ppe_adj_ms = e0.elapsed_time(e1)
    # the reverse of one step with respect to the velocities against one forward
    # step of the same workload (the reverse re-assembles the step's operators)
    s_f, s_b = vct.Solver(sc), vct.Solver(sc)
    st_f, st_b = vct.DeviceState(sc), vct.DeviceState(sc)
    vb = torch.randn((2, sc.n), dtype=torch.float64, device="cuda", generator=g)
    xb = torch.randn((2, sc.n), dtype=torch.float64, device="cuda", generator=g)
    ks = min(args.steps, 10)
    step_ms = timed(lambda: s_f.vct_step(st_f, 1), ks)
    sbw_ms = timed(lambda: s_b.vct_step_backward_velocity(st_b, vb, xb), ks)
    _, sst = s_b.vct_step_backward_velocity(st_b, vb, xb)
    # the workload's loss (squared levels at 8 gauges, the step's free-surface
    # flags) after one step, and its gradient with respect to the starting
    # velocities: forward step + loss against forward step + loss + position
    # gradient + step reverse
    gauges = np.linspace(2.0, 8.0, 8)
    fs = s_b.vct_step_probe(st_b.clone())[0]["fs"]
    st1 = st_b.clone()

    def loss_only():
        for k in vct.DeviceState.FIELDS:   # one step on from st_b's state
            getattr(st1, k).copy_(getattr(st_b, k))
        s_f.vct_step(st1, 1)
        return s_f.vct_gauge_loss(st1, fs, gauges, grad=False)

    def loss_and_grad():
        loss_only()
        _, _, pos_bar = s_f.vct_gauge_loss(st1, fs, gauges)
        return s_b.vct_step_backward_velocity(st_b, None, pos_bar, None)

    fwd_loss_ms = timed(loss_only, ks)
    grad_ms = timed(loss_and_grad, ks)
    # the same reverse on the 2-D wave (45k particles), whose steps run the particle
    # regularisation: the reverse then replays the step forward up to it first
    sw = S.solitary_sigma(precision=args.precision)
    w_f, w_b = vct.Solver(sw), vct.Solver(sw)
    wst_f, wst_b = vct.DeviceState(sw), vct.DeviceState(sw)
    wvb = torch.randn((2, sw.n), dtype=torch.float64, device="cuda", generator=g)
    wave_step_ms = timed(lambda: w_f.vct_step(wst_f, 1), ks)
    wave_bwd_ms = timed(lambda: w_b.vct_step_backward_velocity(wst_b, wvb), ks)
    # and on the 3-D beach slice (702,810 particles, aspect 4, regularisation on)
    s3 = S.beach_bfe_3d(L=8.0, W=1.6, precision=args.precision)
    b_f, b_b = vct.Solver(s3), vct.Solver(s3)
    bst_f, bst_b = vct.DeviceState(s3), vct.DeviceState(s3)
    bvb = torch.randn((3, s3.n), dtype=torch.float64, device="cuda", generator=g)
    k3 = min(ks, 3)
    slice_step_ms = timed(lambda: b_f.vct_step(bst_f, 1), k3)
    slice_bwd_ms = timed(lambda: b_b.vct_step_backward_velocity(bst_b, bvb), k3)
    print(json.dumps({"metric": "adjoint/forward time, one step (its reverse with respect to "
                                "the velocities)",
                      "value": sbw_ms / step_ms, "unit": "x", "higher_is_better": False,
                      "forward_ms": step_ms, "backward_ms": sbw_ms, "calls": ks, "n_gpus": 1,
                      "data": "synthetic",
                      "dtype": "f32+f64" if args.precision == 1 else "f64",
                      "config": {"workload": WORKLOADS["adjoint"], "n_fluid": sc.n_fluid},
                      "sph2_operator": {"forward_ms": fwd, "adjoint_ms": bwd, "ratio": bwd / fwd,
                                        "fields": 3, "calls": k},
                      "ppe_solve": {"forward_ms": fwd_solve_ms, "adjoint_ms": ppe_adj_ms,
                                    "ratio": ppe_adj_ms / fwd_solve_ms,
                                    "adjoint_iters": int(ast.krylov_iters_total)},
                      "step_velocity": {"forward_step_ms": step_ms, "backward_ms": sbw_ms,
                                        "ratio": sbw_ms / step_ms, "calls": ks,
                                        "adjoint_iters": int(sst.krylov_iters_total)},
                      "step_velocity_regularised": {"workload": "2-D sigma solitary wave, "
                                                                "45k particles, regularisation on",
                                                    "forward_step_ms": wave_step_ms,
                                                    "backward_ms": wave_bwd_ms,
                                                    "ratio": wave_bwd_ms / wave_step_ms},
                      "step_velocity_3d": {"workload": "3-D BFE beach slice 8 x 1.6 m, 702,810 "
                                                       "particles, aspect 4, regularisation on",
                                           "forward_step_ms": slice_step_ms,
                                           "backward_ms": slice_bwd_ms,
                                           "ratio": slice_bwd_ms / slice_step_ms},
                      "gauge_loss_gradient": {"what": "d(gauge loss after one step)/d(starting "
                                                      "velocities), 8 gauges",
                                              "forward_ms": fwd_loss_ms, "gradient_ms": grad_ms,
                                              "ratio": grad_ms / fwd_loss_ms},
                      "scope": "operator adjoint, pressure-solve adjoint and the one-step "
                               "reverse with respect to the velocities (positions held); the "
                               "reverse through the positions, chained over steps, is not "
                               "built"}), flush=True)


def run_efficiency(args):
    """The BF / BFE / sigma efficiency comparison (Sec. 4.4.1, Table fig:s4_s_time)
    on the hydrostatic sine + slope tank: per model the particles, the device
    memory of its context, the time per step, particle-updates/s and the
    relative L2 error of the pressure against hydrostatic after the run.  Not
    the headline line."""
    import numpy as np
    import torch
    from paper_2607_28872_b300 import scenarios as S
    from paper_2607_28872_b300 import vct
    if dist_env()[0] != 0:
        return
    steps = min(args.steps, 400) if args.steps else 400
    rows = {}
    for kind in ("BF", "BFE", "SIGMA"):
        sc = S.efficiency_tank(kind, precision=args.precision)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        solver = vct.Solver(sc)
        state = vct.DeviceState(sc)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        solver.vct_step(state, max(args.warmup, 3))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = solver.vct_step(state, steps)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        g = state.numpy()
        f = sc.type == S.FLUID
        surf = np.sort(g["z"][f])[-1]
        hyd = sc.params["rho"] * sc.params["g"] * (sc.params["H"] - g["z"])
        deep = f & (g["p"] > 0)
        e_l2 = float(np.linalg.norm((g["p"] - hyd)[deep]) / np.linalg.norm(hyd[deep]))
        vmax = float(np.sqrt(g["u"] ** 2 + g["w"] ** 2)[f].max())
        rows[kind] = {"n_fluid": sc.n_fluid, "n_particles": sc.n, "d0": sc.params["d0"],
                      "context_mb": (free0 - free1) / 2 ** 20, "ms_per_step": ms,
                      "particle_updates_per_s": sc.n_fluid / (ms / 1e3),
                      "krylov_iters_per_step": st.krylov_iters_total / steps,
                      "p_rel_l2_err": e_l2, "v_max": vmax, "top_z": float(surf)}
        solver.close()
        del state
    bf = rows["BF"]
    for kind in rows:
        rows[kind]["particles_vs_bf"] = rows[kind]["n_fluid"] / bf["n_fluid"]
        rows[kind]["time_vs_bf"] = rows[kind]["ms_per_step"] / bf["ms_per_step"]
    print(json.dumps({"metric": "BF / BFE / sigma efficiency on the hydrostatic sine + slope tank",
                      "steps": steps, "dt": 5e-4, "n_gpus": 1, "data": "synthetic",
                      "dtype": "f32+f64" if args.precision == 1 else "f64",
                      "config": {"workload": WORKLOADS["efficiency"]}, "models": rows}), flush=True)


# schedule table of the ensemble (paper_2607_28872_b300/autotune.py), measured on a B300
TUNING_TABLE = os.path.join(ROOT, "paper_2607_28872_b300", "tuning", "ensemble_b300.json")


def run_ensemble(args):
    """Ensemble throughput through vct_batch_step (not the headline line)."""
    import torch
    from paper_2607_28872_b300 import scenarios as S
    from paper_2607_28872_b300 import vct
    if dist_env()[0] != 0:   # one line per job: rank 0's (replicas only)
        return
    scs = S.ensemble(n_scen=args.ensemble_size, precision=args.precision)
    nf = sum(sc.n_fluid for sc in scs)
    from paper_2607_28872_b300 import autotune
    table, schedule = None, "built-in defaults"
    if args.tune:
        # the batch runs the large-system form above 75k particles in total
        # every class in the large-system form with the batch's V(0,1) cycle: timed
        # alone, V(1,1) wins some classes by a few per cent, side by side it
        # loses (the batch is bandwidth-bound where a single solve is not)
        table = autotune.tune(scs, form=2,
                              grid=lambda dim, form: autotune.candidates(dim, form, cycles=(2,)))
        autotune.save(table, args.tune)
        schedule = f"autotuned now ({len(table)} size classes, written to {args.tune})"
    elif not args.no_tuning and os.path.exists(TUNING_TABLE):
        table = autotune.load(TUNING_TABLE)
        schedule = f"autotuned table {os.path.relpath(TUNING_TABLE, ROOT)} ({len(table)} size classes)"
    knobs = [autotune.tuned(sc, table) if table else {} for sc in scs]
    solvers = [vct.Solver(sc, **kn) for sc, kn in zip(scs, knobs)]
    states = [vct.DeviceState(sc) for sc in scs]
    # every scenario is a wave with the 2-D wave's stable horizon: time at most 100 steps
    steps, warmup = min(args.steps, 100), max(args.warmup, 3)
    warmup += warmup % 2   # an even warm-up leaves the buffers in the parity the timed call starts in,
    #                        so that its pairs replay the graph the warm-up captured
    vct.vct_batch_step(solvers, states, warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    e0.record()
    stats = vct.vct_batch_step(solvers, states, steps)
    e1.record()
    e1.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # end to end: the states in pinned host memory, every step's inputs copied to the
    # device, one vct_batch_step of one step, the states read back
    hosts = [{k: getattr(st, k).cpu().pin_memory() for k in vct.DeviceState.FIELDS}
             for st in states]
    nbytes = sum(t.numel() * t.element_size() for h in hosts for t in h.values())
    ke = min(steps, 10)
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record()
    for _ in range(ke):
        for st, h in zip(states, hosts):
            for k, t in h.items():
                getattr(st, k).copy_(t, non_blocking=True)
        vct.vct_batch_step(solvers, states, 1)
        for st, h in zip(states, hosts):
            for k, t in h.items():
                t.copy_(getattr(st, k), non_blocking=True)
    e3.record()
    e3.synchronize()
    e2e_ms = e2.elapsed_time(e3) / ke
    e2e = {"value": nf / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "steps": ke, "ms_per_step": e2e_ms,
           "note": "one vct_batch_step of one step per step (no graph replay)"}
    # roofline of the batched solve (one launch per step for all scenarios),
    # timed by the first context's profiling events in a further short call
    # (profiling runs the steps from direct launches)
    nprof = 10
    solvers[0].vct_set_profiling(True)
    pst = vct.vct_batch_step(solvers, states, nprof)
    stage_t = solvers[0].vct_stage_times()   # the batched launches of all scenarios
    k_ms, k_cnt = stage_t["krylov"]
    solvers[0].vct_set_profiling(False)
    per_launch, asm = 0.0, 0.0
    key = (2, args.precision)
    for sc, s in zip(scs, pst):
        box = [sc.box_hi[k] - sc.box_lo[k] for k in range(3)]
        re = sc.params["re_over_l"] * sc.params["l_over_d0"] * sc.params["d0"]
        n_cells = (int(box[0] / re) + 1) * (int(box[2] / re) + 1)
        it = s.krylov_iters_total / nprof
        per_launch += B_IT[key] * sc.n_fluid * it
        asm += krylov_bytes(it, s.ppe_rows, s.ppe_nnz, n_cells, args.precision == 1, sc.dim,
                            s.mg_cycle)
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(pk_path)) if os.path.exists(pk_path) else {}
    hbm = peaks.get("hbm_gbs", 6400.0)
    avg_ms = k_ms / max(k_cnt, 1)
    achieved = per_launch / (avg_ms / 1e3) / 1e9
    roof = {"kernel": "k_krylov_fly_batch", "bound": "hbm", "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "traffic": None, "traffic_source": None,
            "peak_source": "measured" if peaks else "fallback", "avg_launch_ms": avg_ms,
            "algorithmic_bytes_per_launch": per_launch, "launches_timed": k_cnt,
            "bytes_model": f"{B_IT[key]:.0f} B per fluid particle and Krylov iteration, summed "
                           "over the scenarios (mean iterations over the profiled call)",
            "assembled_operator_bytes_per_launch": asm,
            "assembled_operator_frac": asm / (avg_ms / 1e3) / 1e9 / hbm,
            "note": "all scenarios' pressure solves in one cooperative launch per step"}
    print(json.dumps({"metric": METRIC, "value": nf * steps / (ms / 1e3), "unit": UNIT,
                      "n_gpus": 1, "steps": steps, "warmup": warmup,
                      "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
                      "data": "synthetic",
                      "config": {"workload": WORKLOADS["ensemble"], "scenarios": len(scs),
                                 "n_fluid_total": nf, "l2": "not flushed (~3 GB working set)"},
                      "krylov_iters_per_step": sum(s.krylov_iters_total for s in stats) / steps,
                      "gpu_launches": int(sum(s.kernel_launches for s in stats)),
                      "graph_steps": int(stats[0].graph_steps), "roofline": roof,
                      "stage_ms_per_step": {k: v[0] / nprof for k, v in stage_t.items() if v[1]},
                      "schedule": schedule, "e2e": e2e,
                      "dtype": "f32+f64" if args.precision == 1 else "f64", "clocks": clk}),
          flush=True)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic bytes per unit of each stage (compulsory traffic: every array
# read or written once per pass; neighbour re-reads are not counted)
# ---------------------------------------------------------------------------
def krylov_bytes(iters, rows, nnz, n_cells, mixed=True, dim=2, cycle=2):
    """Bytes one multigrid-preconditioned BiCGSTAB launch of the assembled
    (large-system) form moves at least, per unknown row and iteration:
    two operator products, each streaming the row (pcnt 4 + diag 8 + (4 col +
    4 or 8 value) per coefficient); the two V-cycles' fine phases -- cycle 2,
    V(0,1) through the row-cell operator: restriction of the input, then the
    3^d row-cell entries plus row index, cell, D^-1, input and output; cycle
    1, V(1,1): the fine residual and the post-smoothing each stream the row
    again -- and the BiCGSTAB vectors (~24 words of the inner precision).
    Coarse levels: per V-cycle each level-1 cell is read (stencil + 4 vectors)
    in the down and up phases (deeper levels add < 1/3).  Set-up: x, b, the
    operator once (twice with the row-cell operator, which it writes)."""
    w = 4 if mixed else 8
    S = 9 if dim == 2 else 27
    nnz_row = nnz / max(rows, 1)
    row = 12 + (4 + w) * nnz_row
    if cycle == 2:
        per_row_iter = 2 * row + 2 * (4 * S + 16 + 3 * w) + 24 * w
        setup = 16 + 12 + 2 * (4 + w) * nnz_row + 4 * S
    else:
        per_row_iter = 6 * row + 30 * w
        setup = 16 + 12 + (4 + w) * nnz_row
    per_cell_iter = 2 * 2 * (S + 4) * 4 * 4 / 3
    return rows * (iters * per_row_iter + setup) + n_cells * iters * per_cell_iter


# Algorithmic bytes per fluid particle of one step, B_step = B_fixed + n_it * B_it
# (n_it = Krylov iterations of the step): compulsory traffic of a matrix-free
# step that reads and writes every per-particle array once per pass (state
# sort/reorder, map and gather records, pass 1, pass 2 + predictor, pressure
# set-up, corrector + update + Jbar) and, per iteration, two matrix-free
# operator products (~68 B each) plus the BiCGSTAB vectors (~96 B).
B_FIXED = {(2, 1): 510.0, (2, 0): 650.0, (3, 1): 800.0, (3, 0): 1000.0}
B_IT = {(2, 1): 230.0, (2, 0): 260.0, (3, 1): 300.0, (3, 0): 360.0}


def fma_peaks():
    """FP32 and FP64 FMA throughput of this GPU (TFLOP/s), measured by a plain
    FMA loop (libvct_peaks.so) timed with CUDA events."""
    import ctypes as C
    from paper_2607_28872_b300 import build
    if not os.path.exists(build.PEAKS_LIB):
        return None
    lib = C.CDLL(build.PEAKS_LIB)
    lib.vct_fma_peak.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    out = {}
    for name, fp64, iters in (("fp32_tflops", 0, 4000), ("fp64_tflops", 1, 200)):
        tf, ms = C.c_double(0), C.c_double(0)
        rc = lib.vct_fma_peak(fp64, iters, C.byref(tf), C.byref(ms))
        out[name] = tf.value if rc == 0 else None
        out[name.replace("tflops", "ms")] = ms.value if rc == 0 else None
    out["how"] = "148x8 blocks x 256 threads x 8 FMA chains, CUDA events, one launch after one warm-up"
    return out


def precision_errors(sc, vct):
    """Error of the mixed form against the FP64 form, per field, after one step
    from the same state (normwise: max |mixed - fp64| / max |fp64| over fluid
    particles).  The mixed step takes the FP64 step's free-surface flags, so
    both solve the same pressure system."""
    import numpy as np
    out = {}
    runs = {}
    fs = None
    for prec in (0, 1):
        s = vct.Solver(sc, precision=prec)
        st = vct.DeviceState(sc)
        pr, _ = s.vct_step_probe(st, fs_in=fs)
        if prec == 0:
            fs = pr["fs"].clone()
        runs[prec] = ({k: v.cpu().numpy() for k, v in pr.items()}, st.numpy())
        s.close()
        del st
    f = sc.type == 0
    g0, s0 = runs[0]
    g1, s1 = runs[1]

    def err(a, b):
        d = np.abs(b).max()
        return float(np.abs(a - b).max() / d) if d > 0 else float(np.abs(a).max())

    for k in ("lam_min", "rho_hat", "nu", "ppe_b"):
        out[k] = err(g1[k][f], g0[k][f])
    for c in range(sc.dim):
        out[f"vstar{c}"] = err(g1["vstar"][c][f], g0["vstar"][c][f])
    for k in ("p", "u", "w") + (("v",) if sc.dim == 3 else ()):
        out[k] = err(s1[k][f], s0[k][f])
    return out


def stage_bytes(stage, n, nf, dim, rows, nnz, nbr_row):
    m = 3 if dim == 2 else 6
    d = dim
    if stage == "pass1":   # reads pos^, pos, vel, type, J, jbar, nbr list; writes L, gv, Ct, rho, lam, fs, nu
        return nf * (8 * (3 * d + 3) + 4 + 4 * nbr_row + 8 * (2 * d * d + d * m + 3) + 4)
    if stage == "pass2":   # reads L, Ct, gv, nu, pos^, vel, metric; writes acc, v*, coefficients
        # (diagonal, wall right side and its d coefficients, counts)
        return nf * (8 * (2 * d * d + d * m + 1 + 2 * d + 4) + 4 * nbr_row + 8 * 3 * d
                     + 12 * (nnz / max(rows, 1)) + 8 * 3 + 4)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_2607_28872_b300 import vct

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sc = workload(args.precision, args.workload)
    n_fluid = sc.n_fluid
    cpu_base = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu_base = cpu_baseline_sample(args.workload, sc)

    solver = vct.Solver(sc)
    # the workloads' trajectories stay well-posed for a limited number of steps
    # (the 2-D wave to ~350, the 3-D beach to ~20: an instability of the
    # stabilised pressure equation at the bottom boundary under high aspect
    # ratios, in the oracle alike): longer runs start again from the initial
    # state every `horizon` steps, outside the timed brackets
    horizon = (150 if sc.dim == 2 else 15) if args.horizon is None else args.horizon
    run = {"state": vct.DeviceState(sc), "since": 0, "total": 0}

    def fresh():
        if horizon and run["since"] >= horizon:
            run["state"] = vct.DeviceState(sc)
            run["since"] = 0
            torch.cuda.synchronize()
        run["since"] += 1
        run["total"] += 1
        return run["state"]

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        solver.vct_step(fresh(), 1)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    total_ms = 0.0
    iters = 0
    launches = 0
    graph_steps = 0
    last = None
    for _ in range(args.steps):
        state = fresh()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            st = solver.vct_step(state, 1)
        except vct.VCTError as err:
            print(f"step {run['total']} of the run failed: {err}", file=sys.stderr, flush=True)
            raise
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        iters += st.krylov_iters_total
        launches += st.kernel_launches
        graph_steps += st.graph_steps
        last = st
    torch.cuda.synchronize()
    clk = clocks.stop()
    # stage times from a further pass of the same steps with the context's stage
    # events on (the events replace the step graphs by direct launches there)
    nprof = max(1, min(args.steps, 30))
    iters_prof = 0
    solver.vct_set_profiling(True)
    for _ in range(nprof):
        state = fresh()
        flush.zero_()
        iters_prof += solver.vct_step(state, 1).krylov_iters_total
    torch.cuda.synchronize()
    stages = solver.vct_stage_times()
    solver.vct_set_profiling(False)
    total_ms = job_ms(total_ms, world)
    ms_step = total_ms / args.steps
    value = job_throughput(n_fluid, world, args.steps, total_ms)

    # e2e: the host-buffer entry point, copies in and out inside the timed region
    e2e = None
    e2e_steps = min(args.steps, 20) if args.e2e_steps is None else args.e2e_steps
    if horizon:   # one fresh run of the workload, within its horizon
        e2e_steps = min(e2e_steps, horizon - 1)
    if rank == 0 and e2e_steps > 0:
        s2 = vct.Solver(sc)
        host = vct.HostState(sc, pin=True)
        s2.vct_step_host(host, 1)
        k = e2e_steps
        t0 = time.perf_counter()
        for _ in range(k):
            s2.vct_step_host(host, 1)
        dt = time.perf_counter() - t0
        narr = 6 if sc.dim == 2 else 8
        e2e = {"value": n_fluid * k / dt, "unit": UNIT,
               "h2d_bytes_per_step": narr * 8 * sc.n + 4 * sc.n,
               "d2h_bytes_per_step": narr * 8 * sc.n}
        s2.close()

    # roofline of the dominant stage (the pressure solve): algorithmic bytes per
    # launch = B_it per fluid particle and iteration x fluid particles x the
    # launch's iterations, over the launch's mean duration (stage events)
    dom = max(stages.items(), key=lambda kv: kv[1][0])
    name, (ms, cnt) = dom
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = peaks.get("hbm_gbs", 6400.0)
    key = (sc.dim, args.precision)
    rows, nnz = last.ppe_rows, last.ppe_nnz
    avg_ms = ms / max(cnt, 1)
    it_launch = iters_prof / max(cnt, 1)
    if name == "krylov":
        per_launch = B_IT[key] * n_fluid * it_launch
    else:
        per_launch = stage_bytes(name, sc.n, n_fluid, sc.dim, rows, nnz, 20 if sc.dim == 2 else 56)
    achieved = per_launch / (avg_ms / 1e3) / 1e9 if per_launch else None
    # the assembled-operator form this solver runs: its own compulsory bytes
    box = [sc.box_hi[k] - sc.box_lo[k] for k in range(3)]
    re = sc.params["re_over_l"] * sc.params["l_over_d0"] * sc.params["d0"]
    n_cells = 1
    for k in range(3):
        if sc.dim == 2 and k == 1:
            continue
        n_cells *= int(box[k] / re) + 1
    asm_bytes = krylov_bytes(it_launch, rows, nnz, n_cells, args.precision == 1, sc.dim,
                             last.mg_cycle)
    traffic, traffic_src = None, None
    tr = NCU_TRAFFIC.get(args.workload)
    if tr and name == "krylov" and args.precision == 1:
        kind, val, traffic_src = tr
        traffic = val if kind == "per_launch" else val * n_fluid * it_launch
    # the solver form the context ran (reported by the library)
    fly = last.solve_form == 1
    roof = {"kernel": {"krylov": "k_krylov_mg_fly" if fly else "k_krylov_mg"}.get(name, name),
            "bound": "hbm",
            "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
            "traffic_source": traffic_src,
            "peak_source": "measured" if peaks else "fallback",
            "avg_launch_ms": avg_ms, "algorithmic_bytes_per_launch": per_launch,
            "bytes_model": f"{B_IT[key]:.0f} B per fluid particle and Krylov iteration "
                           f"x {n_fluid} x {it_launch:.2f} iterations per launch",
            "assembled_operator_bytes_per_launch": asm_bytes,
            "assembled_operator_frac": asm_bytes / (avg_ms / 1e3) / 1e9 / hbm}
    n_it = iters / args.steps
    b_step = B_FIXED[key] + n_it * B_IT[key]
    step_gbs = b_step * n_fluid / (ms_step / 1e3) / 1e9
    step_roof = {"bytes_per_fluid_particle": b_step, "achieved": step_gbs, "peak": hbm,
                 "unit": "GB/s", "frac": step_gbs / hbm,
                 "model": f"{B_FIXED[key]:.0f} + {B_IT[key]:.0f} x {n_it:.2f} iterations"}
    errs = None
    if rank == 0 and not args.no_fp64_probe and args.precision == 1:
        errs = precision_errors(sc, vct)
    pk = fma_peaks() if rank == 0 else None
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == 1 else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n_fluid": n_fluid, "n_particles": sc.n,
                       "dt": sc.params["dt"], "krylov_rtol": sc.params["krylov_rtol"],
                       "l2": ("flushed before every timed step (256 MB write)" if sc.n < 1_000_000 else
                              "inputs larger than L2 (~10 GB working set); also flushed before every "
                              "timed step (256 MB write)"),
                       "parallelism": f"replicas x{world}"},
            "krylov_iters_per_step": iters / args.steps,
            "stage_ms_per_step": {k: v[0] / nprof for k, v in stages.items()},
            "stage_times": f"{nprof} further steps with stage events (direct launches)",
            "graph_steps": graph_steps,
            "roofline": roof, "step_roofline": step_roof, "cpu_baseline": cpu_base, "e2e": e2e,
            "mixed_vs_fp64_err": errs, "fma_peaks": pk,
            "gpu_launches": launches, "clocks": clk}
    print(json.dumps(line), flush=True)


def _oracle_time(sc, nsteps):
    from oracle import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    st = O.OracleState(sc)
    t0 = time.perf_counter()
    st, info = O.step(sc, st, nsteps=nsteps, rtol=sc.params["krylov_rtol"])
    dt = time.perf_counter() - t0
    return dt, cores, info


def sample_scenario(name, sc, precision=1):
    """A bounded sample of the workload for the oracle (about 10-30 s of host
    work per step): the full scenario when it is small, else a slice."""
    from paper_2607_28872_b300 import scenarios as S
    if sc.n_fluid <= 100_000:
        return sc, f"the full {sc.n_fluid}-fluid-particle workload"
    if name in ("beach_bfe_3d", "beach_bfe_3d_slice"):
        sub = S.beach_bfe_3d(L=2.0, W=0.6, x0=1.0, precision=precision)
        return sub, (f"a 2 x 0.6 m slice of the 3-D beach ({sub.n_fluid} fluid particles, "
                     f"same d0, aspect and depth)")
    return sc, f"the full {sc.n_fluid}-fluid-particle workload"


def cpu_baseline_sample(name, sc, nsteps=1):
    """The oracle as it stands, one step of a bounded sample on the host cores."""
    sub, what = sample_scenario(name, sc, sc.params["precision"])
    dt, cores, info = _oracle_time(sub, nsteps)
    return {"value": sub.n_fluid * nsteps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nsteps} step of {what} ({dt:.1f} s, BiCGSTAB rtol "
                      f"{sub.params['krylov_rtol']:g})"}


def reference_sample(name, steps_total, precision, budget_s=150.0):
    """A slice of the workload sized so that steps_total oracle steps take about
    budget_s on the host cores (measured oracle rates: ~4e3 particle-updates/s
    for the 3-D beach, ~2.5e4 for the 2-D channel, on 16 cores)."""
    from paper_2607_28872_b300 import scenarios as S
    if name in ("beach_bfe_3d", "beach_bfe_3d_slice"):
        target = budget_s * 4.0e3 / max(steps_total, 1)          # fluid particles
        L = min(4.0, max(0.4, target / 44000.0))                  # ~44k fluid per m at W = 0.3 m
        sc = S.beach_bfe_3d(L=L, W=0.3, x0=0.5 * L, precision=precision)
        return sc, f"{L:.2f} x 0.30 m slice of the 3-D beach ({sc.n_fluid} fluid particles)"
    full_step_s = 8.0          # measured order of one oracle step on the full 10 m channel
    frac = min(1.0, max(0.08, budget_s / (steps_total * full_step_s)))
    L = 10.0 * frac
    sc = S.solitary_sigma(L=L, bump_x=0.5 * L, x0=0.2 * L, precision=precision)
    return sc, f"channel slice L={L:.2f} m ({sc.n_fluid} fluid particles) of the 10 m workload"


def run_reference(args):
    """The oracle (FP64 CPU reference) on the host cores, a bounded slice of the
    workload per step so that --steps K --warmup W ends within a few minutes."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    sc, what = reference_sample(args.workload, args.steps + args.warmup, args.precision,
                                args.ref_budget)
    from oracle import oracle as O
    cores = O.set_threads(os.cpu_count() or 1)
    st = O.OracleState(sc)
    if args.warmup:
        st, _ = O.step(sc, st, nsteps=args.warmup, rtol=sc.params["krylov_rtol"])
    t0 = time.perf_counter()
    st, info = O.step(sc, st, nsteps=args.steps, rtol=sc.params["krylov_rtol"])
    dt = time.perf_counter() - t0
    value = sc.n_fluid * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS.get(args.workload, args.workload),
                       "n_fluid": sc.n_fluid, "sample": what},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{what}, {args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "efficiency":
        run_efficiency(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
