"""Benchmark: critical-curve roots/s on GB300 (whole hot path per step).

A step is one pass of the full path over one synthetic field: field set-up
(cc_field_create), critical curves on the phi grid with the fused polish and caustic
mapping (cc_critical_curves), the caustic-crossing map (cc_crossing_map) and the
distance-to-caustic map (cc_distance_map).  The default workload is N = 1000 stars
(log-uniform masses in [0.08, 1] rescaled to mean 1, kappa_* = 0.4, kappa_s = 0,
gamma = 0.4), m = 10^4 phi steps (20 002 000 critical points), 4096^2 maps over +-10.

Metric: roots/s = (m+1) * n_r / step time, each root certified to < 1e-9 theta_*
(polish error estimate, see cc_field_report).  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torch.distributed.run: every rank solves its own replica of the
workload (one process per GPU, no data-path collective), timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "critical-curve roots/s at 1e-9 theta_E (batched/served vs plain FP64); p99 latency"
UNIT = "roots/s"

# FP32 pipe operations (FADD, FMUL, FFMA each counted once) of the FP32 tracer (the dominant
# kernel once the polish uses local expansions), csrc/aberth.cu: per star term summed
# directly (acc_star), per root-root term (acc_root), and per evaluation of a cell's two
# 14-term local expansions with the first two derivatives (13 Horner steps of 4 complex
# multiply-adds, 16 FP32 ops each).
TRACE_OPS_PER_STAR = 21
TRACE_OPS_PER_ROOT = 6
TRACE_OPS_PER_FAR_EVAL = 13 * 16


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["n1000", "small"], default="n1000")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain-fp64", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU work for the oracle sample")
    p.add_argument("--msteps", type=int, default=0, help="override the phi steps m (smaller profiling runs)")
    p.add_argument("--map", type=int, default=0, help="override the map size (pixels per side)")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-served", action="store_true")
    p.add_argument("--batched-fields", type=int, default=64)
    p.add_argument("--batched-m", type=int, default=1000)
    p.add_argument("--served-requests", type=int, default=48)
    p.add_argument("--root-refresh", type=int, default=None,
                   help="FP32 tracer: exact far part of the Aberth root sum every K warm rows (0 = exact in "
                        "every sweep; default: the library's)")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(backend: str):
    import torch.distributed as dist
    world, rank, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return world, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def workload(name, msteps=0, pixels=0):
    from paper_2506_02121_gb300 import synth
    wl = synth.workload_n1000() if name == "n1000" else synth.workload_small()
    if msteps:
        wl.msteps = int(msteps)
    if pixels:
        wl.map_pixels = int(pixels)
    if msteps or pixels:
        wl.name = f"{wl.name.split('_')[0]}_m{wl.msteps}_map{wl.map_pixels}"
    return wl


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args):
    import numpy as np
    import torch

    world, rank = init_dist("nccl" if args.gpus > 1 else "gloo")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2506_02121_gb300 import cc

    wl = workload(args.workload, args.msteps, args.map)
    f = wl.fields[0]
    m = wl.msteps
    ext, px = wl.map_extent, wl.map_pixels
    pixel = 2 * ext / px
    xs = torch.from_numpy(f.x).to(dev)
    ys = torch.from_numpy(f.y).to(dev)
    ms = torch.from_numpy(f.m).to(dev)
    nr = 2 * f.n
    rows = m + 1
    roots_per_step = rows * nr

    # outputs and scratch, allocated once
    fopt = cc.cc_options_default()
    if args.root_refresh is not None:
        fopt.root_refresh = args.root_refresh
    probe = cc.cc_field_create(xs, ys, ms, f.kappa_s, f.gamma, fopt)
    ws_cc = cc.workspace(cc.cc_critical_curves_workspace_bytes(probe, m), dev)
    del probe
    z = torch.empty((rows, nr), dtype=torch.complex128, device=dev)
    w = torch.empty_like(z)
    ncc = torch.empty((px, px), dtype=torch.int32, device=dev)
    dmap = torch.empty((px, px), dtype=torch.float64, device=dev)
    ws_d = cc.workspace(cc.cc_distance_map_workspace_bytes(px, px), dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)
    launches_per_step = 0

    def step():
        """Enqueue one step on the stream; returns the field, the stage events and an event
        recorded after the step's last kernel (the field is released, and its report read,
        only after that event: neither is part of the step's work)."""
        nonlocal launches_per_step
        field = cc.cc_field_create(xs, ys, ms, f.kappa_s, f.gamma, fopt)
        cc.cc_critical_curves(field, m, z, w, None, ws_cc, stream)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
              torch.cuda.Event(enable_timing=True))
        ev[0].record(stream)
        cc.cc_crossing_map(w, -ext, ext, -ext, ext, px, px, ncc, stream)
        ev[1].record(stream)
        cc.cc_distance_map(ncc, pixel, dmap, ws_d, stream)
        ev[2].record(stream)
        end = torch.cuda.Event(enable_timing=True)
        end.record(stream)
        return field, ev, end

    def report(field):
        nonlocal launches_per_step
        status, rep = cc.cc_field_report(field)
        S = rep["subchains"]
        # phase table, tracer, seam match (S > 1), permutation compose; polish stage (far field:
        # extent, setup, occupancy, slots, coefficients, point kernel, direct kernel that
        # returns at once; else the direct kernel); rescue; crossing scatter + row scan;
        # distance map feature, chunk, column and row kernels
        polish_kernels = 7 if f.n >= 128 else 1
        launches_per_step = 1 + 1 + (1 if S > 1 else 0) + 1 + polish_kernels + 1 + 2 + 4
        return status, rep

    for _ in range(args.warmup):
        fld, _, end = step()
        end.synchronize()
        report(fld)
        del fld
    torch.cuda.synchronize()

    timers = []
    step_ms = []
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t_wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1)  # L2 flush between timed steps (outside the step's events)
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fld, ev, e1 = step()
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            status, rep = report(fld)
            timers.append((rep, ev, status))
            del fld
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t_wall0
    clocks = clk.summary()

    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_step = total_ms / args.steps
    value = world * roots_per_step * args.steps / (total_ms / 1e3)

    reps = [t[0] for t in timers]
    status_ok = all(t[2] == cc.CC_OK for t in timers)
    rep = reps[-1]
    polish_ms = statistics.mean(r["polish_ms"] for r in reps)
    trace_ms = statistics.mean(r["trace_ms"] for r in reps)
    join_ms = statistics.mean(r["join_ms"] for r in reps)
    cross_ms = statistics.mean(t[1][0].elapsed_time(t[1][1]) for t in timers)
    dist_ms = statistics.mean(t[1][1].elapsed_time(t[1][2]) for t in timers)

    peaks, peak_src = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tops = 152 * 128 * sm_max * 1e6 / 1e12  # FP32 lane-ops per second at max clock
    trace_ops = (rep["star_terms"] * TRACE_OPS_PER_STAR + rep["root_terms"] * TRACE_OPS_PER_ROOT
                 + rep["far_evals"] * TRACE_OPS_PER_FAR_EVAL)
    stage = {"trace_ms": trace_ms, "join_ms": join_ms, "polish_caustic_ms": polish_ms,
             "crossing_ms": cross_ms, "distance_ms": dist_ms}
    achieved = trace_ops / (trace_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "trace_kernel<float> (FP32 Aberth tracer, dominant stage)",
                "achieved": round(achieved, 3), "peak": round(fp32_peak_tops, 3), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak_tops, 4), "traffic": None,
                "peak_source": f"152 SMs x 128 FP32 lanes x {sm_max:.0f} MHz (FP32 pipe ops, FADD/FMUL/FFMA = 1)",
                "ops_per_unit": {"star_term": TRACE_OPS_PER_STAR, "root_term": TRACE_OPS_PER_ROOT,
                                 "far_eval": TRACE_OPS_PER_FAR_EVAL},
                "units": f"{rep['star_terms']} star terms, {rep['root_terms']} root terms "
                         f"({rep['root_iterations']} root-iterations), {rep['far_evals']} expansion evaluations"}
    # crossing map: algorithmic bytes = vertex reads + one int32 read+write per pixel for
    # the scan + the clearing store
    cross_bytes = rows * nr * 16 + 3 * px * px * 4
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    extra = {
        "polish": {"ms": round(polish_ms, 3), "passes": rep["polish_passes"],
                   "method": "local expansions (32 terms) for stars beyond a 5x5 block of cells, direct double-float "
                             "sums for the rest"},
        "crossing_map": {"achieved_gbs": round(cross_bytes / (cross_ms / 1e3) / 1e9, 1),
                         "frac_hbm": round(cross_bytes / (cross_ms / 1e3) / 1e9 / hbm, 4)},
    }

    out = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
        "config": {"workload": wl.name, "n_stars": f.n, "n_roots": nr, "phi_steps": m,
                   "root_points_per_step": roots_per_step, "map": f"{px}x{px} over +-{ext}",
                   "kappa_star": f.kappa_star, "kappa_s": f.kappa_s, "gamma": f.gamma,
                   "subchains": rep["subchains"], "root_refresh": fopt.root_refresh,
                   "l2": "flushed (256 MiB write) between timed steps",
                   "precision": "FP32 Aberth tracer + double-float certified polish/caustics; FP64 segment tests"},
        "roofline": roofline,
        "stages_ms": {k: round(v, 3) for k, v in stage.items()},
        "kernels": extra,
        "accuracy": {"max_err_est": rep["max_err_est"], "uncertified": rep["uncertified"],
                     "unconverged": rep["unconverged"], "status_ok": status_ok,
                     "polish_passes_per_point": round(rep["polish_passes"] / roots_per_step, 4),
                     "tracer_iterations_per_point": round(rep["root_iterations"] / roots_per_step, 4),
                     "jumped": rep["jumped"], "rescued": rep["rescued_points"]},
        "clocks": clocks,
        "gpu_launches": launches_per_step * args.steps,
        "wall_s": round(wall, 3),
    }
    if not args.no_plain_fp64 and rank == 0:
        out["plain_fp64"] = plain_fp64(args, f, m, dev, xs, ys, ms, roots_per_step)
    if not args.no_e2e:
        out["e2e"] = e2e(args, f, m, ext, px, pixel, dev, world)
    if not args.no_batched and rank == 0:
        out["batched"] = batched(args, dev)
    if not args.no_served and rank == 0:
        out["served"] = served(args, dev)
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(f, m, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out))
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()


def plain_fp64(args, f, m, dev, xs, ys, ms, roots_per_step):
    """The same workload with the plain FP64 tracer (|dz| < 1e-9 stop rule) and FP64 caustics."""
    import torch
    from paper_2506_02121_gb300 import cc
    o = cc.cc_options_default()
    o.precision = cc.CC_FP64
    o.hp_arith = cc.CC_HP_FP64
    field = cc.cc_field_create(xs, ys, ms, f.kappa_s, f.gamma, o)
    ws = cc.workspace(cc.cc_critical_curves_workspace_bytes(field, m), dev)
    rows, nr = m + 1, 2 * f.n
    z = torch.empty((rows, nr), dtype=torch.complex128, device=dev)
    w = torch.empty_like(z)
    stream = torch.cuda.current_stream(dev)
    cc.cc_critical_curves(field, m, z, w, None, ws, stream)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cc.cc_critical_curves(field, m, z, w, None, ws, stream)
    e1.record(stream)
    e1.synchronize()
    ms_ = e0.elapsed_time(e1)
    st, rep = cc.cc_field_report(field)
    del ws, z, w
    torch.cuda.empty_cache()
    return {"value": round(roots_per_step / (ms_ / 1e3), 1), "unit": UNIT, "ms": round(ms_, 2), "steps": 1,
            "warmup": 1, "trace_ms": round(rep["trace_ms"], 2), "caustic_ms": round(rep["polish_ms"], 2),
            "status_ok": st == cc.CC_OK, "note": "critical curves + caustics only (no maps), FP64 Aberth"}


def e2e(args, f, m, ext, px, pixel, dev, world):
    """Same metric through the public API with host buffers: star arrays from pinned host
    memory in, critical points, caustics and both maps back to pinned host memory."""
    import numpy as np
    import torch
    from paper_2506_02121_gb300 import cc
    rows, nr = m + 1, 2 * f.n
    hx = torch.from_numpy(f.x).pin_memory()
    hy = torch.from_numpy(f.y).pin_memory()
    hm = torch.from_numpy(f.m).pin_memory()
    hz = torch.empty((rows, nr), dtype=torch.complex128).pin_memory()
    hw = torch.empty_like(hz).pin_memory()
    hn = torch.empty((px, px), dtype=torch.int32).pin_memory()
    hd = torch.empty((px, px), dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream(dev)

    copy_stream = torch.cuda.Stream(dev)

    def once():
        field = cc.cc_field_create(hx, hy, hm, f.kappa_s, f.gamma)
        z, w, _ = cc.critical_curves(field, m, caustics=True, stream=stream)
        # the critical points and caustics are final here: copy them back on a second stream
        # while the maps are computed
        ready = torch.cuda.Event()
        ready.record(stream)
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):
            hz.copy_(z, non_blocking=True)
            hw.copy_(w, non_blocking=True)
        z.record_stream(copy_stream)
        w.record_stream(copy_stream)
        ncc = cc.crossing_map(w, -ext, ext, -ext, ext, px, px, stream)
        d = cc.distance_map(ncc, pixel, stream)
        hn.copy_(ncc, non_blocking=True)
        hd.copy_(d, non_blocking=True)
        torch.cuda.synchronize()

    once()
    steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        once()
    el = max_over_ranks(time.perf_counter() - t0, dev)
    h2d = 3 * 8 * f.n
    d2h = hz.numel() * 16 + hw.numel() * 16 + hn.numel() * 4 + hd.numel() * 8
    return {"value": round(world * rows * nr * steps / el, 1), "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def batched(args, dev):
    """Many fields in one persistent launch replayed as a CUDA graph: a sample of the
    batched workload (fields with N log-uniform in [50, 5000], unit masses, kappa_* in
    U[0.1, 0.8], gamma in U[0, 0.8], kappa_s in U[0, 0.3]), tile shape from the autotuner."""
    import torch
    from paper_2506_02121_gb300 import autotune, cc, synth
    wl = synth.workload_batched(args.batched_fields, args.batched_m)
    fopt = cc.cc_options_default()
    if args.root_refresh is not None:
        fopt.root_refresh = args.root_refresh
    fields = [cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, fopt) for f in wl.fields]
    ms = [wl.msteps] * len(fields)
    t, items, info = autotune.tune(fields, ms, probe_steps=32, repeats=1)
    b = cc.cc_batch_create(fields, ms, t, items)
    z = [torch.empty((m + 1, fl.n_roots), dtype=torch.complex128, device=dev) for fl, m in zip(fields, ms)]
    w = [torch.empty_like(a) for a in z]
    ws = cc.workspace(cc.cc_batch_workspace_bytes(b), dev)
    cc.cc_batch_bind(b, z, w, ws)
    stream = torch.cuda.Stream(dev)
    cc.cc_batch_launch(b, True, stream)  # capture + first replay (warm-up)
    stream.synchronize()
    times = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cc.cc_batch_launch(b, True, stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    st, per, tot = cc.cc_batch_report(b)
    roots = sum((m + 1) * fl.n_roots for fl, m in zip(fields, ms))
    ms_ = min(times)
    ninfo = cc.cc_batch_info(b)
    del z, w, ws
    torch.cuda.empty_cache()
    return {"value": round(roots / (ms_ / 1e3), 1), "unit": UNIT, "ms": round(ms_, 2), "fields": len(fields),
            "phi_steps": wl.msteps, "roots": roots, "items": ninfo["items"], "grid": ninfo["grid"],
            "block_threads": t, "items_per_cta": items, "tuned_from_cache": info["cached"],
            "status_ok": st == cc.CC_OK, "max_err_est": tot["max_err_est"],
            "stages_ms": {"trace": round(tot["trace_ms"], 2), "join": round(tot["join_ms"], 2),
                          "polish_caustic": round(tot["polish_ms"], 2)},
            "workload": f"{len(fields)} fields of the batched distribution (N log-U[50,5000]), m={wl.msteps}, "
                        f"one persistent launch replayed from a CUDA graph"}


def served(args, dev):
    """Continuous-batching server on a Poisson trace (50 req/s) of critical-curve + caustic +
    1024^2 crossing-map requests with N log-uniform in [100, 20000], m = 200."""
    import torch
    from paper_2506_02121_gb300 import synth
    from paper_2506_02121_gb300.serve import GpuExecutor, Request, Server, summarize
    reqs = []
    for i, (t, f) in enumerate(synth.served_requests(args.served_requests, 50.0)):
        reqs.append(Request(rid=i, arrival=t, x=f.x, y=f.y, mass=f.m, kappa_s=f.kappa_s, gamma=f.gamma,
                            msteps=200, map_extent=10.0, map_pixels=1024))
    slots = 4
    srv = Server(GpuExecutor(slots=slots, device=dev.index or 0), slots=slots, budget_bytes=96 << 30)
    warm = Server(GpuExecutor(slots=1, device=dev.index or 0), slots=1, budget_bytes=96 << 30)
    warm.run([reqs[0]], realtime=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = srv.run(reqs, realtime=True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    st = summarize(res, wall)
    out = {"value": round(st["roots_per_s"], 1) if st["roots_per_s"] else None, "unit": UNIT,
           "p50_latency_s": round(st["p50_s"], 4) if st["p50_s"] is not None else None,
           "p99_latency_s": round(st["p99_s"], 4) if st["p99_s"] is not None else None,
           "requests": st["requests"], "ok": st["ok"], "errors": st["errors"], "noconv": st["noconv"],
           "slots": slots, "arrival_rate_hz": 50.0, "wall_s": round(wall, 3),
           "workload": "Poisson 50 req/s, N log-U[100,20000], log-U masses, m=200, 1024^2 maps over +-10"}
    del srv
    torch.cuda.empty_cache()
    return out


def cpu_baseline(f, m, seconds):
    """The FP64 oracle on this host's cores, on a bounded sample of the same workload:
    warm-started rows after the centre row (Aberth + Newton polish + caustic mapping of
    each row), scaled to roots/s."""
    import numpy as np
    import oracle
    c = m // 2
    z, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(c, m))  # untimed seed
    rows = 0
    t0 = time.perf_counter()
    while True:
        j = c + 1 + rows
        z, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, m), z0=z)
        oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, z)
        rows += 1
        if time.perf_counter() - t0 > seconds or rows >= 200:
            break
    el = time.perf_counter() - t0
    nr = 2 * f.n
    return {"value": round(rows * nr / el, 1), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{rows} warm-started rows (phi_j, j = m/2+1..m/2+{rows}) of the {f.n}-star field: "
                      f"Aberth + Newton polish + caustic mapping, {el:.1f} s"}


def run_reference(args):
    """Reference arm: the FP64 oracle (the only reference implementation of this method)
    timed as it stands on the host cores, each step a bounded sample of the workload."""
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import oracle
    wl = workload(args.workload, args.msteps, args.map)
    f = wl.fields[0]
    m = wl.msteps
    nr = 2 * f.n
    c = m // 2
    z, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(c, m))
    rows_per_step = 20
    times = []
    j = c
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _ in range(rows_per_step):
            j += 1
            z, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, m), z0=z)
            oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, z)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = rows_per_step * nr * args.steps / total
    sample = (f"{rows_per_step} warm-started rows per step of the {f.n}-star, m={m} field "
              f"(Aberth + Newton polish + caustic mapping), FP64 oracle")
    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "n_stars": f.n, "n_roots": nr, "phi_steps": m},
           "impl": "reference",
           "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
