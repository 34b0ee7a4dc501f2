#!/usr/bin/env python
"""Throughput of the ERPP coupling step on GB300.

One step = bin + gather + self-disturbance removal + Stokes drag + FP64
Euler advance + regularised source scatter (erpp_step), FP32 kernels with
FP64 particle integration, on the homogeneous-shear-like workload: periodic
box 4pi x 2pi x 2pi, 512 x 256 x 256 grid, 1,000,000 particles, sigma_R = dx,
stencil radius 3 sigma_R, mean shear S = 1, Stokes-number mix {0.1, 1, 10},
mass loading 0.4.  The fluid field is held fixed (the fluid solver is not
part of the coupling step).  Inputs are synthetic and seeded.

Metric: particle-stencil node updates per second (every stencil node of
every particle, counted once for the gather and once for the scatter), and
coupling steps per second.  With --gpus N > 1 (torchrun) every rank runs an
independent box of its own (weak scaling, no data-path collective).

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import erpp_inputs as I  # noqa: E402

WORKLOAD = I.CFG_SHEAR
METRIC = "particle-stencil node updates/s (gather + scatter) at 1M particles"
UNIT = "node-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kahan", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tile shape instead of timing the candidates")
    ap.add_argument("--tiling", default=None,
                    help="fixed tile shape TYxTZ[xTHREADS] (for example 32x2x256) instead of "
                         "the autotuner")
    ap.add_argument("--scatter-mode", default=None, choices=["merge", "cluster", "xclip"],
                    help="with --tiling: how tile halos reach their neighbours (default merge)")
    ap.add_argument("--no-loop", action="store_true",
                    help="skip the closed-loop (coupling + fluid stand-in) timing")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the timing of the PIC and point-value-gather steps")
    ap.add_argument("--weights", default="gaussian", choices=["gaussian", "pic", "point"],
                    help="time the step with other weights (pic: trilinear particle-in-cell; "
                         "point: 4-point Lagrange point-value gather) instead of the ERPP "
                         "kernel; the extra timings are then skipped")
    ap.add_argument("--full-force", action="store_true",
                    help="time the step with the general force of Eq. force_particle "
                         "(ERPP_FULL_FORCE: Faxen, added mass, one-step Basset memory); the "
                         "extra timings are then skipped")
    ap.add_argument("--lag", action="store_true",
                    help="time the step with the source delayed by eps_R (ERPP_LAG: "
                         "round(eps_R/dt) steps of positions and forces kept on the device); "
                         "the extra timings are then skipped")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra records (compensated scatter, 256^3 box, 64 batched "
                         "boxes)")
    ap.add_argument("--workload", default="shear", choices=["shear", "cube256", "batched64"],
                    help="shear: 512x256x256 box (the benchmark); cube256: 256^3, 1M "
                         "particles (profiling case); batched64: 64 independent boxes "
                         "(64^3-128^3, 1e3-2e5 particles each) stepped as one graph")
    return ap.parse_args()


def dist_env():
    from paper_1405_6969_gb300 import dist as D
    return D.env()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed loop runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        loaded = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def stencil_nodes(x, w):
    """Stencil nodes per particle (same window rule as the kernels), summed."""
    sig = math.sqrt(2 * w.nu * w.eps_R)
    rc = w.cutoff * sig
    total = np.ones(x.shape[1], dtype=np.int64)
    for a in range(3):
        inv = w.n[a] / w.L[a]
        s = x[a] * inv
        cp = rc * inv
        total *= (np.floor(s + cp) - np.ceil(s - cp) + 1).astype(np.int64)
    return int(total.sum())


def algorithmic_bytes(w, n_p):
    """Bytes the step must move: read u and write S once
    (12 B per node each, FP32), and per particle read x, v, x_prev, D,
    radius, rho_p (112 B) and write x, v, x_prev, D (96 B)."""
    return {"gather": 12 * w.n_nodes, "scatter": 12 * w.n_nodes, "advance": 208 * n_p,
            "step": 24 * w.n_nodes + 208 * n_p}


def captured_traffic(w, kernel, tiling, mode):
    """DRAM bytes (read + write) per launch of the dominant phase from the ncu
    capture summarised in profiles/, when it was taken on this workload, tile
    shape, halo mode and kernel source; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "erpp_step_shear512_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        with open(os.path.join(ROOT, d["source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError, KeyError):
        return None
    if (d.get("workload") != w.name or kernel != "scatter" or sha != d.get("source_sha256")
            or list(tiling[2:5]) != list(d.get("tiling", [])) or mode not in d.get("modes", {})):
        return None
    return d["modes"][mode]["traffic_bytes"]


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = WORKLOAD
    grid, _ = I.make_grid(w)
    st = I.make_particles(w, None)
    n_s = 20000
    p = w.params()
    times = []
    nodes = 0
    for k in range(args.warmup + args.steps):
        sub = I.ParticleState(*(np.ascontiguousarray(a[..., (k * n_s) % w.n_particles:][..., :n_s])
                                for a in (st.x, st.v, st.x_prev, st.D, st.radius, st.rho_p)))
        nn = 2 * stencil_nodes(sub.x, w)
        t0 = time.perf_counter()
        oracle.step(p, grid, sub, first_step=False)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
            nodes += nn
    total = sum(times)
    value = nodes / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "particles_per_step_sample": n_s,
                   "grid": list(w.n), "box": list(w.L)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n_s} particles of the 1M cloud per step on the full "
                                   f"512x256x256 grid (one oracle step each)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def cpu_baseline(w, grid, st, gpu_step=None):
    """The FP64 oracle timed on the host cores on a bounded sample (500k of
    the particles, full grid).  gpu_step(sample) -> {mode: (S, D, v)} runs the
    GPU step on the same sample; its error against this oracle step is
    returned too (the oracle runs here and nowhere else in the bench)."""
    import oracle
    oracle.build()
    n_s = 500_000
    sub = I.ParticleState(*(np.ascontiguousarray(a[..., :n_s])
                            for a in (st.x, st.v, st.x_prev, st.D, st.radius, st.rho_p)))
    inp = sub.copy()
    nn = 2 * stencil_nodes(sub.x, w)
    t0 = time.perf_counter()
    S_ref = oracle.step(w.params(), grid, sub, first_step=False)
    dt = time.perf_counter() - t0
    errors = None
    if gpu_step is not None:
        errors = {"sample": f"one step of {n_s} of the particles on the full grid, against "
                            f"this oracle step", "tolerance": 1e-5}
        for mode, (S, D, v) in gpu_step(inp).items():
            errors[mode] = {"S": rel_l2(S, S_ref), "D": rel_l2(D, sub.D), "v": rel_l2(v, sub.v)}
    del S_ref
    out = {"value": nn / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"one FP64 oracle step of {n_s} of the 1M particles on the full "
                     f"512x256x256 grid ({dt:.1f} s, single thread)"}
    # The same sample on every host core: the unchanged oracle step on one particle
    # chunk per thread, partial sources summed over z-slabs (oracle.step_threads).
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    if cores and cores > 1:
        sub = I.ParticleState(*(np.ascontiguousarray(a[..., :n_s])
                                for a in (st.x, st.v, st.x_prev, st.D, st.radius, st.rho_p)))
        t0 = time.perf_counter()
        oracle.step_threads(w.params(), grid, sub, cores, first_step=False)
        dt_all = time.perf_counter() - t0
        out["all_cores"] = {"value": nn / dt_all, "cores": cores,
                            "sample": f"the same step on {cores} threads ({dt_all:.2f} s, "
                                      f"{dt / dt_all:.1f}x the single thread)"}
    return out, errors


def batched_record(args, ws, rank, steps, peak):
    """64 independent boxes: one replayed CUDA graph per step, against the
    same boxes as 64 plain launch sequences and against the plain FP64 form.
    Returns the record (rank 0) with the timings, the step's HBM roofline
    and the FP32 batched result's difference from the FP64 plain form on one
    step of every box (the FP64 form matches the FP64 oracle to 1e-12)."""
    import torch
    from paper_1405_6969_gb300 import Batch, ParticleState
    from paper_1405_6969_gb300 import dist as D
    boxes = I.batched_boxes(64, seed0=D.batched_seed0(rank))
    nodes_per_step = 0
    made = []
    for w in boxes:
        grid, _ = I.make_grid(w)
        st = I.make_particles(w, None)
        nodes_per_step += 2 * stencil_nodes(st.x, w)
        made.append((w, grid, st))

    def batch(precision):
        dt = torch.float32 if precision == "fp32" else torch.float64
        entries = []
        for w, grid, st in made:
            u = torch.as_tensor(grid, dtype=dt).cuda().contiguous()
            entries.append((w.params(), u, ParticleState.from_numpy(st), torch.empty_like(u)))
        return Batch(entries, precision=precision), entries

    stream = torch.cuda.current_stream()
    warm = max(3, args.warmup)

    def timed(b, use_graph, nsteps):
        for k in range(warm):
            b.step(first_step=(k == 0), use_graph=use_graph)
        b.check()
        D.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nsteps):
            b.step(use_graph=use_graph)
        e1.record(stream)
        torch.cuda.synchronize()
        D.barrier()
        b.check()
        return D.max_over_ranks(e0.elapsed_time(e1) / nsteps, device="cuda")

    # accuracy at the timed configuration: one step (not a first step) of
    # every box from the same state, FP32 batched graph against FP64 plain
    b32, e32 = batch("fp32")
    tiles = None
    if not args.no_autotune:
        import collections
        cache = os.path.join(tempfile.mkdtemp(), "tune.json")
        tiles = collections.Counter("x".join(map(str, t)) if t else "x-halo"
                                    for t in b32.autotune(cache_path=cache))
    b64, e64 = batch("fp64")
    b32.step(first_step=False, use_graph=True)
    b64.step(first_step=False, use_graph=False)
    b32.check()
    b64.check()
    num = {"S": 0.0, "D": 0.0, "v": 0.0}
    den = {"S": 0.0, "D": 0.0, "v": 0.0}
    for (_, _, p32, S32), (_, _, p64, S64) in zip(e32, e64):
        for k, (a32, a64) in {"S": (S32, S64), "D": (p32.D, p64.D),
                              "v": (p32.v, p64.v)}.items():
            num[k] += float(((a32.double() - a64) ** 2).sum())
            den[k] += float((a64 ** 2).sum())
    accuracy = {k: math.sqrt(num[k] / max(den[k], 1e-300)) for k in num}
    b32.close()
    b64.close()
    del e32, e64

    b32, _ = batch("fp32")
    if tiles:
        b32.autotune(cache_path=cache)  # the cached choices: no timing
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms_graph = timed(b32, True, steps)
    clocks = sampler.stop()
    launches_per_step = b32.last_step_launches()  # the graph's kernels
    ms_eager = timed(b32, False, max(3, steps // 4))
    # the other graph form: nine kernels over all boxes (persistent gather and
    # scatter over (box, tile) work items)
    b32.set_form("multi")
    ms_multi = timed(b32, True, steps)
    multi_launches = b32.last_step_launches()
    b32.set_form("branches")
    b32.close()
    b64, _ = batch("fp64")
    ms_f64 = timed(b64, False, max(3, min(steps // 10, 10)))
    b64.close()
    torch.cuda.empty_cache()
    value = D.aggregate_rate(nodes_per_step, ws, ms_graph * 1e-3)
    if rank != 0:
        return None
    n_p = sum(w.n_particles for w, _, _ in made)
    n_nodes = sum(w.n_nodes for w, _, _ in made)
    alg = 24 * n_nodes + 208 * n_p
    achieved = alg / (ms_graph * 1e-3) / 1e9
    return {
        "metric": "particle-stencil node updates/s (gather + scatter), 64 batched boxes",
        "value": value, "unit": UNIT, "n_gpus": ws, "steps": steps,
        "warmup": warm, "ms_per_step": ms_graph, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 kernels, f64 particle integration", "data": "synthetic",
        "config": {"workload": "batched64_boxes_64-128cube_1e3-2e5_particles",
                   "boxes": len(made), "particles_total": n_p, "nodes_total": n_nodes,
                   "l2": "inputs larger than L2 (about 0.9 GB of grids)"},
        "steps_per_s": 1e3 / ms_graph,
        "plain_launches_ms_per_step": ms_eager,
        "graph_speedup_vs_plain_launches": ms_eager / ms_graph,
        "multi_box_form": {"ms_per_step": ms_multi, "gpu_launches_per_step": multi_launches,
                           "note": "the same step as nine kernels over all boxes "
                                   "(erpp_batch_set_form multi)"},
        "fp64_plain_form_ms_per_step": ms_f64,
        "speedup_vs_fp64_plain_form": ms_f64 / ms_graph,
        "accuracy_fp32_vs_fp64_plain": dict(accuracy, tolerance=1e-5,
                                            note="relative L2 over all boxes of one step; "
                                                 "both forms meet the 1e-5 stated accuracy "
                                                 "when these are below it"),
        "tiles_per_box": dict(tiles) if tiles else None,
        "roofline": {"bound": "hbm", "kernel": "whole batched step (graph)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "alg_bytes": alg},
        "gpu_launches": launches_per_step * steps,
        "clocks": clocks,
    }


def run_batched(args, ws, rank, local):
    import torch
    import torch.distributed as dist
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peak, peak_kind = measured_peaks()
    line = batched_record(args, ws, rank, args.steps, peak)
    if rank == 0:
        line["roofline"]["peak_kind"] = peak_kind
        line["cpu_baseline"] = None
        line["e2e"] = None
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


PHASES = ["bin", "gather", "advance", "scatter"]


def workload_record(w, args, peak, kahan=False, steps=100, made=None):
    """One more single-box workload (the same step, its own autotuned tiles):
    ms per step, node updates/s, per-phase times and the HBM roofline of the
    slower tile phase and of the whole step.  made: (u, particle state) of
    the workload when already on hand."""
    import torch
    from paper_1405_6969_gb300 import Context, ParticleState
    if made is None:
        grid64, _ = I.make_grid(w)
        st = I.make_particles(w, None)
        u = torch.as_tensor(grid64, dtype=torch.float32).cuda().contiguous()
        del grid64
    else:
        u, st = made
    ps = ParticleState.from_numpy(st)
    ctx = Context(w.params(), precision="fp32", kahan=kahan)
    S = ctx.new_grid()
    if args.tiling:
        t = [int(v) for v in args.tiling.lower().split("x")] + [0]
        ctx.set_tiling(t[0], t[1], t[2])
        if args.scatter_mode:
            ctx.set_scatter_mode(args.scatter_mode)
    elif not args.no_autotune:
        from paper_1405_6969_gb300 import autotune
        autotune.tune(ctx, u, ps, S=S, use_cache=False)
    stream = torch.cuda.current_stream()
    for k in range(max(3, args.warmup)):
        ctx.step(u, ps, S=S, first_step=(k == 0))
    ctx.check()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.step(u, ps, S=S)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.check()
    # per-phase times in steps of their own (no events between the timed
    # steps' kernels)
    ctx.profile_enable(True)
    ctx.profile_read()
    for _ in range(min(steps, 50)):
        ctx.step(u, ps, S=S)
    phase_ms, nsteps = ctx.profile_read()
    ctx.profile_enable(False)
    ctx.check()
    ms = e0.elapsed_time(e1) / steps
    nodes = 2 * stencil_nodes(st.x, w)
    per = {nm: phase_ms[k] / max(nsteps, 1) for k, nm in enumerate(PHASES)}
    alg = algorithmic_bytes(w, w.n_particles)
    dom = max(("gather", "scatter"), key=lambda nm: per[nm])
    ach = alg[dom] / (per[dom] * 1e-3) / 1e9
    step_gbs = alg["step"] / (ms * 1e-3) / 1e9
    rec = {"workload": w.name, "grid": list(w.n), "particles": w.n_particles,
           "kahan": bool(kahan), "ms_per_step": ms, "steps": steps,
           "node_updates_per_s": nodes / (ms * 1e-3), "steps_per_s": 1e3 / ms,
           "phase_ms": per, "tiling": ctx.tiling(),
           "roofline": {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak,
                        "unit": "GB/s", "frac": ach / peak, "traffic": None},
           "step_hbm": {"alg_bytes": alg["step"], "achieved_gbs": step_gbs,
                        "frac": step_gbs / peak},
           "gpu_launches_per_step": ctx.last_step_launches()}
    ctx.close()
    del u, S, ps
    torch.cuda.empty_cache()
    return rec


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batched64":
        import torch
        torch.cuda.set_device(local)
        from paper_1405_6969_gb300 import build as libbuild
        libbuild.build()
        run_batched(args, ws, rank, local)
        return
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1405_6969_gb300 import Context, ParticleState
    from paper_1405_6969_gb300 import build as libbuild
    libbuild.build()

    w = WORKLOAD if args.workload == "shear" else I.CFG_CUBE256
    from paper_1405_6969_gb300 import dist as D
    seed = D.box_seed(0, rank)
    grid64, _ = I.make_grid(w, seed=w.field_seed + seed)
    st = I.make_particles(w, None, seed=w.particle_seed + seed)
    u = torch.as_tensor(grid64, dtype=torch.float32).cuda().contiguous()
    ps = ParticleState.from_numpy(st)
    ctx = Context(w.params(), precision="fp32", kahan=args.kahan, weights=args.weights,
                  lag=args.lag, full_force=args.full_force)
    S = ctx.new_grid()
    if args.lag or args.full_force or args.kahan or args.workload != "shear":
        args.no_extra = True
    if args.lag or args.full_force:
        args.no_loop = args.no_e2e = args.no_cpu_baseline = args.no_variants = True
    if args.weights == "gaussian":
        nodes_per_step = 2 * stencil_nodes(st.x, w)
    else:
        args.no_extra = True
        args.no_loop = args.no_e2e = args.no_cpu_baseline = args.no_variants = True
        nodes_per_step = (16 * w.n_particles if args.weights == "pic"
                          else 64 * w.n_particles + stencil_nodes(st.x, w))
    stream = torch.cuda.current_stream()

    # tile shape: time the candidates on this workload (a few steps each, on
    # copies of the particle state) and keep the fastest
    tiling = {"tiling": ctx.tiling()}
    if args.tiling:
        t = [int(v) for v in args.tiling.lower().split("x")] + [0]
        ctx.set_tiling(t[0], t[1], t[2])
        if args.scatter_mode:
            ctx.set_scatter_mode(args.scatter_mode)
        tiling = {"tile": tuple(t[:3]), "mode": ctx.scatter_mode(), "tiling": ctx.tiling(),
                  "ms": None, "cached": False}
    elif args.lag:
        # the first round(eps_R/dt) delayed steps have no source to time: keep
        # the tile shape the autotuner picks for this workload without delay
        ctx.set_tiling(16, 2, 256)
        tiling = {"tile": (16, 2, 256), "tiling": ctx.tiling(), "ms": None, "cached": False}
    elif not args.no_autotune and args.weights != "pic":
        from paper_1405_6969_gb300 import autotune
        tiling = autotune.tune(ctx, u, ps, S=S, use_cache=False)

    # warm-up (the first step has no previous force to remove; with the delayed
    # source, past the round(eps_R/dt) + 1 steps without source or removal)
    warm = args.warmup + (max(1, round(w.eps_R / w.dt)) + 1 if args.lag else 0)
    for k in range(warm):
        ctx.step(u, ps, S=S, first_step=(k == 0))
    ctx.check()
    torch.cuda.synchronize()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.step(u, ps, S=S)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ctx.check()
    # per-phase times from the library's events on the launching stream, in
    # steps of their own (events between the phases would sit between kernels
    # that otherwise launch back to back, so the timed steps above have none)
    ctx.profile_enable(True)
    ctx.profile_read()
    for _ in range(min(args.steps, 50)):
        ctx.step(u, ps, S=S)
    phase_ms, nsteps = ctx.profile_read()
    ctx.profile_enable(False)
    ctx.check()
    # per-step times of 50 more steps, each between its own events: the median
    # (the timed region above gives the mean)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(51)]
    evs[0].record(stream)
    for k in range(50):
        ctx.step(u, ps, S=S)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    ctx.check()
    ms_median = statistics.median(evs[k].elapsed_time(evs[k + 1]) for k in range(50))
    elapsed_ms = e0.elapsed_time(e1)
    t_max = elapsed_ms
    if ws > 1:
        t = torch.tensor([elapsed_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    ms_per_step = t_max / args.steps
    value = ws * nodes_per_step * args.steps / (t_max * 1e-3)

    # roofline of the dominant kernel, timed live with CUDA events (the
    # per-phase events are recorded by the ERPP-kernel step only)
    per = {nm: phase_ms[k] / max(nsteps, 1) for k, nm in enumerate(PHASES)}
    alg = algorithmic_bytes(w, w.n_particles)
    peak, peak_kind = measured_peaks()
    roofline = None
    if nsteps > 0:
        dom = max(("gather", "scatter"), key=lambda nm: per[nm])
        achieved = alg[dom] / (per[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak,
                    "traffic": captured_traffic(w, dom, ctx.tiling(), ctx.scatter_mode()),
                    "peak_kind": peak_kind}
    step_gbs = alg["step"] / (ms_per_step * 1e-3) / 1e9

    # the scatter phase against the measured rate of the shared-memory add it
    # accumulates with: each stencil node of each particle receives one
    # contribution per force component (one 32-bit add, two with the split
    # words of the compensated form)
    atomics = None
    if nsteps > 0 and args.weights == "gaussian":
        from paper_1405_6969_gb300 import shared_add_rate
        peak_s32 = shared_add_rate("s32")
        updates = 3 * (nodes_per_step // 2)
        ach = updates / (per["scatter"] * 1e-3)
        atomics = {"kernel": "scatter phase (accumulation, write-out, halo merges)",
                   "node_component_updates": updates,
                   "adds_per_update": 2 if args.kahan else 1,
                   "achieved_updates_per_s": ach,
                   "peak_adds_per_s": peak_s32,
                   "frac": ach * (2 if args.kahan else 1) / peak_s32,
                   "peak_fp32_adds_per_s": shared_add_rate("f32"),
                   "peak_kind": "measured live: shared-memory 32-bit atomic add, conflict-free "
                                "lanes, every SM full (erpp_shared_add_rate)"}

    # the closed loop of the shear workload: coupling step, then the fluid
    # stand-in forced by the new source (the fluid is timed on its own too)
    loop = None
    if not args.no_loop:
        from paper_1405_6969_gb300 import StokesFluid
        fl = StokesFluid(w.params(), precision="fp32")
        u_loop = u.clone()
        for _ in range(3):
            fl.step(u_loop, S)
        l0 = torch.cuda.Event(enable_timing=True)
        l1 = torch.cuda.Event(enable_timing=True)
        l2 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        l0.record(stream)
        for _ in range(20):
            fl.step(u_loop, S)
        l1.record(stream)
        n_loop = 100
        lev = [torch.cuda.Event(enable_timing=True) for _ in range(n_loop)]
        for k in range(n_loop):
            ctx.step(u_loop, ps, S=S)
            fl.step(u_loop, S)
            lev[k].record(stream)
        l2.record(stream)
        torch.cuda.synchronize()
        ctx.check()
        fluid_ms = l0.elapsed_time(l1) / 20
        loop_ms = l1.elapsed_time(l2) / n_loop
        per_step = [l1.elapsed_time(lev[0])] + [lev[k - 1].elapsed_time(lev[k])
                                                for k in range(1, n_loop)]
        loop = {"steps": n_loop, "loop_ms_per_step": loop_ms,
                "loop_ms_per_step_median": statistics.median(per_step),
                "fluid_ms_per_step": fluid_ms,
                "coupling_ms_per_step": loop_ms - fluid_ms,
                "fluid": "exact periodic Stokes step (cuFFT R2C/C2R + spectral kernel)"}
        del u_loop
        fl.close()

    # the same workload with the other weights (ERPP_PIC: trilinear source and
    # gather, 8 + 8 nodes per particle; ERPP_POINT_GATHER: 4-point Lagrange
    # gather, 64 nodes, and the Gaussian source)
    variants = None
    if not args.no_variants:
        variants = {}
        for kind in ("pic", "point"):
            vctx = Context(w.params(), precision="fp32", weights=kind)
            vps = ParticleState.from_numpy(st)
            for k in range(3):
                vctx.step(u, vps, S=S, first_step=(k == 0))
            torch.cuda.synchronize()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            n_var = 50
            v0.record(stream)
            for _ in range(n_var):
                vctx.step(u, vps, S=S)
            v1.record(stream)
            torch.cuda.synchronize()
            vctx.check()
            v_ms = v0.elapsed_time(v1) / n_var
            nodes = (16 * w.n_particles if kind == "pic"
                     else 64 * w.n_particles + stencil_nodes(st.x, w))
            variants[kind] = {"ms_per_step": v_ms, "node_updates_per_step": nodes,
                              "node_updates_per_s": nodes / (v_ms * 1e-3),
                              "gpu_launches_per_step": vctx.last_step_launches()}
            vctx.close()
            del vps

    # end to end through the public API: host (pinned) buffers in and out
    e2e = None
    if not args.no_e2e:
        # every step: the field and the whole particle state in from pinned
        # host memory, the source and the updated state back (erpp_step_host:
        # the copies of one step overlap the neighbouring steps' computation)
        hu = torch.empty(u.shape, dtype=torch.float32, pin_memory=True).copy_(u.cpu())
        hs = ps.pinned()
        hS = torch.empty(S.shape, dtype=torch.float32, pin_memory=True)
        h2d = hu.numel() * 4 + sum(t.numel() * 8 for t in (hs.x, hs.v, hs.x_prev, hs.D,
                                                           hs.radius, hs.rho_p))
        d2h = hS.numel() * 4 + sum(t.numel() * 8 for t in (hs.x, hs.v, hs.x_prev, hs.D))
        k_e2e = max(3, min(args.steps, 20))
        for _ in range(2):  # staging buffers allocated before the timed steps
            ctx.step_host(hu, hs, hS)
        ctx.step_host_wait()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(k_e2e):
            ctx.step_host(hu, hs, hS)
        ctx.step_host_wait()
        a1.record(stream)
        torch.cuda.synchronize()
        e_ms = a0.elapsed_time(a1)
        if ws > 1:
            t = torch.tensor([e_ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e_ms = float(t.item())
        e2e = {"value": ws * nodes_per_step * k_e2e / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": k_e2e,
               "ms_per_step": e_ms / k_e2e}

    # extra records: the compensated (Kahan) scatter on this workload, the
    # 256^3 / 1M box and the 64 batched boxes, each timed on its own
    extra = {}
    if not args.no_extra:
        extra["kahan"] = workload_record(w, args, peak, kahan=True, steps=50, made=(u, st))
        extra["cube256"] = workload_record(I.CFG_CUBE256, args, peak, steps=100)
        extra["batched64"] = batched_record(args, ws, rank, 20, peak)

    cpu = None
    errors = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        def gpu_step(sample):
            # the timed workload's step (its tiles) on the oracle's sample, in
            # both scatter modes
            out = {}
            for mode in ("fixed_point", "kahan"):
                ectx = Context(w.params(), precision="fp32", kahan=(mode == "kahan"))
                t = ctx.tiling()
                if t[0] == 4:
                    ectx.set_tiling(t[2], t[3], t[4])
                ectx.set_scatter_mode(ctx.scatter_mode())
                eps = ParticleState.from_numpy(sample)
                eS = ectx.step(u, eps, first_step=False)
                ectx.check()
                out[mode] = (eS.cpu().numpy(), eps.D.cpu().numpy(), eps.v.cpu().numpy())
                ectx.close()
                del eS, eps
            return out
        cpu, errors = cpu_baseline(w, grid64, st, gpu_step)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 kernels, f64 particle integration", "data": "synthetic",
            "config": {"workload": w.name, "grid": list(w.n), "box": [round(v, 6) for v in w.L],
                       "particles_per_gpu": w.n_particles, "sigma_over_dx": w.sigma_over_dx,
                       "cutoff_sigmas": w.cutoff, "precision": "fp32",
                       "kahan": bool(args.kahan), "weights": args.weights,
                       "lag_steps": (max(1, round(w.eps_R / w.dt)) if args.lag else 0),
                       "force": "general (Eq. force_particle)" if args.full_force else "Stokes drag",
                       "l2": "inputs larger than L2: u and S 403 MB each, particles 112 MB",
                       "fluid": "held fixed during the timed steps"},
            "steps_per_s": 1e3 / ms_per_step,
            "ms_per_step_median_of_50": ms_median,
            "node_updates_per_step": nodes_per_step,
            "phase_ms": per if nsteps > 0 else None,
            "step_hbm": {"alg_bytes": alg["step"], "achieved_gbs": step_gbs,
                         "frac": step_gbs / peak},
            "roofline": roofline,
            "atomics": atomics,
            "cpu_baseline": cpu,
            "error_vs_oracle": errors,
            "kahan": extra.get("kahan"),
            "cube256": extra.get("cube256"),
            "batched64": extra.get("batched64"),
            "coupled_loop": loop,
            "weights_variants": variants,
            "tiling": tiling,
            "e2e": e2e,
            # counted by the library at each kernel launch of a step
            "gpu_launches": ctx.last_step_launches() * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
