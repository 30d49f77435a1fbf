"""Benchmark: critical-curve roots/s on GB300 (whole hot path per step).

A step is one pass of the full path over one synthetic field: field set-up
(cc_field_create), critical curves on the phi grid with the fused polish and caustic
mapping (cc_critical_curves), the caustic-crossing map (cc_crossing_map) and the
distance-to-caustic map (cc_distance_map).  The default workload is N = 1000 stars
(log-uniform masses in [0.08, 1] rescaled to mean 1, kappa_* = 0.4, kappa_s = 0,
gamma = 0.4), m = 10^4 phi steps (20 002 000 critical points), 4096^2 maps over +-10.

Metric: roots/s = (m+1) * n_r / step time, each root certified to < 1e-9 theta_*
(polish error estimate, see cc_field_report).  Prints one JSON line on rank 0, which also
carries (rank 0, one GPU):
  plain_fp64 / mixed_fp64_polish  the same field by the paper's all-FP64 form and by the
                                  mixed form with a native FP64 polish;
  e2e                             the step from host buffers through the public API;
  batched                         256 fields (N log-uniform in [50, 5000], m = 5000) in one
                                  graph-replayed persistent launch, the same fields solved
                                  one after another, and a spread of them by plain FP64;
  served                          500 Poisson requests (50/s, N up to 20000, m = 200, 1024^2
                                  maps): p50/p99, roots/s, saturation rate, and the first
                                  requests served by the plain FP64 form;
  large_field                     N = 20000, m = 2*10^4, 8192^2 maps, one timed pass;
  cpu_baseline                    the FP64 oracle on the host cores (all and one), scaled
                                  from a sample of the step, with the FP64-oracle error of
                                  every point of the GPU step (accuracy.vs_fp64_oracle).

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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "critical-curve roots/s at 1e-9 theta_E (batched/served vs plain FP64); p99 latency"
UNIT = "roots/s"

# FP32 pipe operations (FADD, FMUL, FFMA each counted once, a packed FP32x2 operation twice)
# of the FP32 tracer (the dominant kernel), csrc/aberth.cu: per star term summed directly
# (acc_star), per root-root term (acc_root), and per evaluation of a cell's 14-term local
# expansions of U and S1' with the derivative chain (far_eval: 13 Horner steps of 8 packed
# FMAs, 16 FP32 ops each).
TRACE_OPS_PER_STAR = 21
TRACE_OPS_PER_ROOT = 6
TRACE_OPS_PER_FAR_EVAL = 13 * 16
# DRAM bytes (read + write) per launch of the tracer on the default workload, from one ncu
# capture of this kernel version (dram__bytes_read.sum 4 021 504 + dram__bytes_write.sum
# 298 724 864, one launch at m = 10^4); to be set to None whenever the kernel changes.
TRACE_TRAFFIC = 302746368


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
    p.add_argument("--no-large", action="store_true", help="skip the N = 20000, m = 2*10^4, 8192^2 line")
    p.add_argument("--no-accuracy", action="store_true", help="skip the FP64-oracle check of every point")
    p.add_argument("--batched-fields", type=int, default=256)
    p.add_argument("--batched-m", type=int, default=5000)
    p.add_argument("--served-requests", type=int, default=500)
    p.add_argument("--compare-fields", type=int, default=8,
                   help="batched fields also solved by the plain FP64 form (spread over the N range)")
    p.add_argument("--compare-requests", type=int, default=8,
                   help="first requests of the served trace also served by the plain FP64 form")
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


def fp_peaks(dev):
    """Measured FP32 and FP64 FMA rates of this GPU (csrc/probe_peaks.cu: grids of
    independent FMA chains), in tera lane-operations per second."""
    import ctypes
    import torch
    from paper_2506_02121_gb300 import build
    lib = ctypes.CDLL(build.build_probe())
    lib.ccprobe_fma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double)]
    lib.ccprobe_fma_rate.restype = ctypes.c_double
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = sms * 8, 256
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    res = {}
    for kind, name, iters in ((0, "ffma_tops", 20000), (1, "ffma2_tops", 10000), (2, "dfma_tops", 400)):
        ops = ctypes.c_double()
        best = 0.0
        for _ in range(3):
            ms = lib.ccprobe_fma_rate(kind, blocks, threads, iters, ctypes.c_void_p(out.data_ptr()), ctypes.byref(ops))
            if ms > 0:
                best = max(best, ops.value / (ms / 1e3) / 1e12)
        res[name] = round(best, 3)
    del out
    return res


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
        # extent, setup, occupancy, slots, coefficients, sub-cells, point kernel, direct kernel that
        # returns at once; else the direct kernel); rescue; crossing scatter + row scan;
        # distance map feature, chunk, column and row kernels
        polish_kernels = 8 if f.n >= 128 else 1
        launches_per_step = 1 + 1 + (1 if S > 1 else 0) + 1 + polish_kernels + 1 + 2 + 4
        return status, rep

    peaks_fp = fp_peaks(dev)
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
    fp32_measured = max(peaks_fp.get("ffma_tops", 0.0), peaks_fp.get("ffma2_tops", 0.0))
    trace_ops = (rep["star_terms"] * TRACE_OPS_PER_STAR + rep["root_terms"] * TRACE_OPS_PER_ROOT
                 + rep["far_evals"] * TRACE_OPS_PER_FAR_EVAL)
    stage = {"trace_ms": trace_ms, "join_ms": join_ms, "polish_caustic_ms": polish_ms,
             "crossing_ms": cross_ms, "distance_ms": dist_ms}
    achieved = trace_ops / (trace_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "trace_kernel<float> (FP32 Aberth tracer, dominant stage)",
                "achieved": round(achieved, 3), "peak": round(fp32_peak_tops, 3), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak_tops, 4), "traffic": TRACE_TRAFFIC,
                "peak_source": f"152 SMs x 128 FP32 lanes x {sm_max:.0f} MHz (FP32 pipe ops, FADD/FMUL/FFMA = 1)",
                "measured_fp32_peak": fp32_measured,
                "frac_of_measured_fp32": round(achieved / fp32_measured, 4) if fp32_measured else None,
                "ops_per_unit": {"star_term": TRACE_OPS_PER_STAR, "root_term": TRACE_OPS_PER_ROOT,
                                 "far_eval": TRACE_OPS_PER_FAR_EVAL},
                "units": f"{rep['star_terms']} star terms, {rep['root_terms']} root terms "
                         f"({rep['root_iterations']} root-iterations, {rep['cold_root_iterations']} of them at "
                         f"cold-started rows), {rep['far_evals']} expansion evaluations"}
    # crossing map: vertex reads + one int32 read+write per pixel for the scan + the clearing
    # store; distance map: N_cc read, g written and read, distance written (8 B)
    cross_bytes = rows * nr * 16 + 3 * px * px * 4
    dist_bytes = px * px * (4 + 4 + 4 + 8)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    extra = {
        "polish": {"ms": round(polish_ms, 3), "passes": rep["polish_passes"],
                   "method": "stars beyond a 5x5 block of cells by local expansions (32 terms per cell, re-centred "
                             "to 16 at each occupied 4x4 sub-cell), direct double-float sums for the rest"},
        "crossing_map": {"bytes": cross_bytes, "achieved_gbs": round(cross_bytes / (cross_ms / 1e3) / 1e9, 1),
                         "frac_hbm": round(cross_bytes / (cross_ms / 1e3) / 1e9 / hbm, 4)},
        "distance_map": {"bytes": dist_bytes, "achieved_gbs": round(dist_bytes / (dist_ms / 1e3) / 1e9, 1),
                         "frac_hbm": round(dist_bytes / (dist_ms / 1e3) / 1e9 / hbm, 4)},
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
        "fp_peaks_measured": peaks_fp,
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
    # the last step's results, for the FP64-oracle error of every point (after all GPU work)
    host = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline and args.no_accuracy):
        host = {"z": z.cpu().numpy(), "w": w.cpu().numpy(), "ncc": ncc.cpu().numpy(), "d": dmap.cpu().numpy()}
    del z, w, ncc, dmap, ws_cc, ws_d, flush
    torch.cuda.empty_cache()
    if not args.no_plain_fp64 and rank == 0:
        out["plain_fp64"] = plain_fp64(args, f, m, dev, xs, ys, ms, roots_per_step)
        out["mixed_fp64_polish"] = mixed_fp64_polish(args, f, m, dev, xs, ys, ms, roots_per_step)
    if not args.no_e2e:
        out["e2e"] = e2e(args, f, m, ext, px, pixel, dev, world)
    if not args.no_batched and rank == 0:
        out["batched"] = batched(args, dev)
    if not args.no_served and rank == 0:
        out["served"] = served(args, dev)
    if not args.no_large and rank == 0 and args.workload == "n1000" and not args.msteps:
        out["large_field"] = large_field(args, dev)
    if host is not None:
        cpu = cpu_baseline(f, m, ext, px, args.cpu_seconds, host)
        if not args.no_accuracy:
            out["accuracy"]["vs_fp64_oracle"] = cpu.pop("accuracy")
        else:
            cpu.pop("accuracy", None)
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out))
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()


def _solve_timed(field, m, dev, stream, caustics=True, warm=True):
    """One warm-up (warm) and one timed cc_critical_curves of a field (CUDA events on stream)."""
    import torch
    from paper_2506_02121_gb300 import cc
    rows = m + 1
    z = torch.empty((rows, field.n_roots), dtype=torch.complex128, device=dev)
    w = torch.empty_like(z) if caustics else None
    ws = cc.workspace(cc.cc_critical_curves_workspace_bytes(field, m), dev)
    if warm:
        cc.cc_critical_curves(field, m, z, w, None, ws, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cc.cc_critical_curves(field, m, z, w, None, ws, stream)
    e1.record(stream)
    e1.synchronize()
    st, rep = cc.cc_field_report(field)
    return e0.elapsed_time(e1), st, rep, (z, w, ws)


def plain_fp64(args, f, m, dev, xs, ys, ms, roots_per_step):
    """The same workload with the plain FP64 tracer (|dz| < 1e-9 stop rule) and FP64 caustics."""
    import torch
    from paper_2506_02121_gb300 import cc
    o = cc.cc_options_default()
    o.precision = cc.CC_FP64
    o.hp_arith = cc.CC_HP_FP64
    field = cc.cc_field_create(xs, ys, ms, f.kappa_s, f.gamma, o)
    ms_, st, rep, bufs = _solve_timed(field, m, dev, torch.cuda.current_stream(dev))
    del bufs
    torch.cuda.empty_cache()
    return {"value": round(roots_per_step / (ms_ / 1e3), 1), "unit": UNIT, "ms": round(ms_, 2), "steps": 1,
            "warmup": 1, "trace_ms": round(rep["trace_ms"], 2), "caustic_ms": round(rep["polish_ms"], 2),
            "status_ok": st == cc.CC_OK, "note": "critical curves + caustics only (no maps), FP64 Aberth"}


def mixed_fp64_polish(args, f, m, dev, xs, ys, ms, roots_per_step):
    """The mixed form with native FP64 polish and caustic mapping (hp_arith = FP64) in place
    of double-float: critical curves + caustics of the same field."""
    import torch
    from paper_2506_02121_gb300 import cc
    o = cc.cc_options_default()
    o.hp_arith = cc.CC_HP_FP64
    if args.root_refresh is not None:
        o.root_refresh = args.root_refresh
    field = cc.cc_field_create(xs, ys, ms, f.kappa_s, f.gamma, o)
    ms_, st, rep, bufs = _solve_timed(field, m, dev, torch.cuda.current_stream(dev))
    del bufs
    torch.cuda.empty_cache()
    return {"value": round(roots_per_step / (ms_ / 1e3), 1), "unit": UNIT, "ms": round(ms_, 2), "steps": 1,
            "warmup": 1, "trace_ms": round(rep["trace_ms"], 2), "polish_caustic_ms": round(rep["polish_ms"], 2),
            "max_err_est": rep["max_err_est"], "uncertified": rep["uncertified"], "rescued": rep["rescued_points"],
            "status_ok": st == cc.CC_OK,
            "note": "FP32 tracer + native FP64 polish and caustics; critical curves + caustics only (no maps)"}


def e2e(args, f, m, ext, px, pixel, dev, world):
    """Same metric through the public API with host buffers: star arrays from pinned host
    memory in, critical points, caustics and both maps back to pinned host memory."""
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


def _spread(fields, k):
    """Indices of k fields spread over the N range: the (2i+1)/(2k) quantiles of N."""
    order = sorted(range(len(fields)), key=lambda i: (fields[i].n, i))
    return [order[min(len(order) - 1, (2 * i + 1) * len(order) // (2 * k))] for i in range(k)]


def batched(args, dev):
    """The batched workload: fields with N log-uniform in [50, 5000], unit masses,
    kappa_* in U[0.1, 0.8], gamma in U[0, 0.8], kappa_s in U[0, 0.3], m phi steps each.
    - batched: one persistent launch of all fields, replayed from a CUDA graph, tile shape
      from the autotuner;
    - sequential: the same fields one after another through cc_critical_curves (each
      field's own launch sequence) on one stream;
    - vs plain FP64: fields spread over the N range solved by the plain FP64 form and,
      on the same fields, by the mixed form one at a time and batched."""
    import torch
    from paper_2506_02121_gb300 import autotune, cc, synth
    wl = synth.workload_batched(args.batched_fields, args.batched_m)
    fopt = cc.cc_options_default()
    if args.root_refresh is not None:
        fopt.root_refresh = args.root_refresh
    fields = [cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, fopt) for f in wl.fields]
    ms = [wl.msteps] * len(fields)
    t_tune = time.perf_counter()
    t, items, info = autotune.tune(fields, ms, probe_steps=64, repeats=1)
    t_tune = time.perf_counter() - t_tune
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
    ms_ = statistics.mean(times)
    ninfo = cc.cc_batch_info(b)
    del ws
    cc.cc_batch_destroy(b)
    torch.cuda.empty_cache()

    # the same fields one after another, each through its own cc_critical_curves
    wsz = max(cc.cc_critical_curves_workspace_bytes(fl, m) for fl, m in zip(fields, ms))
    ws1 = cc.workspace(wsz, dev)
    for i in _spread(fields, 4):  # warm-up: every kernel variant loaded
        cc.cc_critical_curves(fields[i], ms[i], z[i], w[i], None, ws1, stream)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for fl, m, zz, ww in zip(fields, ms, z, w):
        cc.cc_critical_curves(fl, m, zz, ww, None, ws1, stream)
    e1.record(stream)
    e1.synchronize()
    seq_ms = e0.elapsed_time(e1)
    seq_ok = all(cc.cc_field_report(fl)[0] == cc.CC_OK for fl in fields)
    del ws1, z, w
    torch.cuda.empty_cache()

    # identical fields through the plain FP64 form, the mixed form one at a time, and batched
    pick = _spread(wl.fields, args.compare_fields)
    sub = [wl.fields[i] for i in pick]
    sub_roots = sum((wl.msteps + 1) * 2 * f.n for f in sub)
    o64 = cc.cc_options_default()
    o64.precision = cc.CC_FP64
    o64.hp_arith = cc.CC_HP_FP64
    fp64_ms = mixed_ms = 0.0
    fp64_ok = mixed_ok = True
    cur = torch.cuda.current_stream(dev)
    for f in sub:
        for opt, which in ((o64, "fp64"), (fopt, "mixed")):
            fl = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, opt)
            el, stt, _, bufs = _solve_timed(fl, wl.msteps, dev, cur, warm=(which == "mixed"))
            del bufs
            if which == "fp64":
                fp64_ms += el
                fp64_ok = fp64_ok and stt == cc.CC_OK
            else:
                mixed_ms += el
                mixed_ok = mixed_ok and stt == cc.CC_OK
    sub_fields = [fields[i] for i in pick]
    bs = cc.batch_critical_curves(sub_fields, [wl.msteps] * len(sub), caustics=True, use_graph=True, stream=stream,
                                  block_threads=t, items_per_cta=items)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cc.cc_batch_launch(bs, True, stream)
    e1.record(stream)
    e1.synchronize()
    sub_batched_ms = e0.elapsed_time(e1)
    sub_st = cc.cc_batch_report(bs)[0]
    del bs
    torch.cuda.empty_cache()
    return {"value": round(roots / (ms_ / 1e3), 1), "unit": UNIT, "ms": round(ms_, 2), "fields": len(fields),
            "phi_steps": wl.msteps, "roots": roots, "items": ninfo["items"], "grid": ninfo["grid"],
            "block_threads": t, "items_per_cta": items, "tuned_from_cache": info["cached"],
            "autotune_s": round(t_tune, 2), "status_ok": st == cc.CC_OK, "max_err_est": tot["max_err_est"],
            "uncertified": tot["uncertified"],
            "stages_ms": {"trace": round(tot["trace_ms"], 2), "join": round(tot["join_ms"], 2),
                          "polish_caustic": round(tot["polish_ms"], 2)},
            "sequential": {"value": round(roots / (seq_ms / 1e3), 1), "ms": round(seq_ms, 2), "status_ok": seq_ok,
                           "batched_speedup": round(seq_ms / ms_, 3),
                           "note": "the same fields one after another, cc_critical_curves per field, one stream"},
            "vs_plain_fp64": {"fields": len(sub), "n_stars": [f.n for f in sub], "roots": sub_roots,
                              "plain_fp64": round(sub_roots / (fp64_ms / 1e3), 1),
                              "mixed_one_at_a_time": round(sub_roots / (mixed_ms / 1e3), 1),
                              "mixed_batched": round(sub_roots / (sub_batched_ms / 1e3), 1),
                              "batched_over_plain_fp64": round(fp64_ms / sub_batched_ms, 1),
                              "status_ok": fp64_ok and mixed_ok and sub_st == cc.CC_OK,
                              "note": "identical fields (the (2i+1)/2k quantiles of N) in every form"},
            "workload": f"{len(fields)} fields of the batched distribution (N log-U[50,5000]), m={wl.msteps}, "
                        f"one persistent launch replayed from a CUDA graph"}


def served(args, dev):
    """Continuous-batching server on a Poisson trace (50 req/s) of critical-curve + caustic +
    1024^2 crossing-map requests with N log-uniform in [100, 20000], m = 200: the whole trace
    in real time, the same requests all at once (saturation throughput), and the first
    requests of the trace served by the plain FP64 form and by the mixed form."""
    import torch
    from paper_2506_02121_gb300 import synth
    from paper_2506_02121_gb300.serve import GpuExecutor, Request, Server, summarize
    reqs = []
    for i, (t, f) in enumerate(synth.served_requests(args.served_requests, 50.0)):
        reqs.append(Request(rid=i, arrival=t, x=f.x, y=f.y, mass=f.m, kappa_s=f.kappa_s, gamma=f.gamma,
                            msteps=200, map_extent=10.0, map_pixels=1024))
    slots = 4
    dev_i = dev.index or 0

    def run(precision, rs, realtime):
        srv = Server(GpuExecutor(slots=slots, device=dev_i, precision=precision), slots=slots,
                     budget_bytes=96 << 30)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = srv.run(rs, realtime=realtime)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st = summarize(res, wall)
        del srv, res
        torch.cuda.empty_cache()
        return st

    def brief(st):
        return {"roots_per_s": round(st["roots_per_s"], 1) if st["roots_per_s"] else None,
                "p50_latency_s": round(st["p50_s"], 4) if st["p50_s"] is not None else None,
                "p99_latency_s": round(st["p99_s"], 4) if st["p99_s"] is not None else None,
                "requests": st["requests"], "ok": st["ok"], "errors": st["errors"], "noconv": st["noconv"],
                "wall_s": round(st["wall_s"], 3)}

    Server(GpuExecutor(slots=1, device=dev_i), slots=1, budget_bytes=96 << 30).run([reqs[0]], realtime=False)
    live = run("mixed", reqs, True)
    sat = run("mixed", reqs, False)
    k = min(args.compare_requests, len(reqs))
    Server(GpuExecutor(slots=1, device=dev_i, precision="fp64"), slots=1,
           budget_bytes=96 << 30).run([reqs[4]], realtime=False)  # warm-up of the FP64 kernels
    fp64 = run("fp64", reqs[:k], True)
    mixed_k = run("mixed", reqs[:k], True)
    span = reqs[-1].arrival
    out = {"value": round(live["roots_per_s"], 1) if live["roots_per_s"] else None, "unit": UNIT,
           "p50_latency_s": brief(live)["p50_latency_s"], "p99_latency_s": brief(live)["p99_latency_s"],
           "requests": live["requests"], "ok": live["ok"], "errors": live["errors"], "noconv": live["noconv"],
           "slots": slots, "arrival_rate_hz": 50.0, "arrival_span_s": round(span, 3), "wall_s": round(live["wall_s"], 3),
           "throughput_req_per_s": round(live["ok"] / live["wall_s"], 2),
           "saturation_req_per_s": round(sat["ok"] / sat["wall_s"], 2),
           "saturated_at_50hz": bool(sat["ok"] / sat["wall_s"] < 50.0),
           "all_at_once": brief(sat),
           "vs_plain_fp64": {"requests": k, "n_stars": [r.n for r in reqs[:k]], "plain_fp64": brief(fp64),
                             "mixed": brief(mixed_k),
                             "mixed_over_plain_fp64_roots_per_s": round(mixed_k["roots_per_s"] / fp64["roots_per_s"], 1)
                             if fp64["roots_per_s"] and mixed_k["roots_per_s"] else None,
                             "note": "the first requests of the same trace, at their arrival times, in both forms"},
           "workload": f"Poisson 50 req/s, {len(reqs)} requests, N log-U[100,20000], log-U masses, m=200, "
                       f"1024^2 maps over +-10"}
    return out


def large_field(args, dev):
    """The largest single field: N = 20000 Kroupa-like stars, kappa_* = 0.2, kappa_s = 0.3,
    gamma = 0.3, m = 2*10^4 phi steps (8.0*10^8 critical points), 8192^2 crossing and distance
    maps over +-10: one warm-up and one timed pass of the whole path."""
    import torch
    from paper_2506_02121_gb300 import cc, synth
    wl = synth.workload_n20000()
    f = wl.fields[0]
    m, ext, px = wl.msteps, wl.map_extent, wl.map_pixels
    xs, ys, mm = (torch.from_numpy(a).to(dev) for a in (f.x, f.y, f.m))
    fopt = cc.cc_options_default()
    if args.root_refresh is not None:
        fopt.root_refresh = args.root_refresh
    probe = cc.cc_field_create(xs, ys, mm, f.kappa_s, f.gamma, fopt)
    nr = probe.n_roots
    ws = cc.workspace(cc.cc_critical_curves_workspace_bytes(probe, m), dev)
    del probe
    z = torch.empty((m + 1, nr), dtype=torch.complex128, device=dev)
    w = torch.empty_like(z)
    ncc = torch.empty((px, px), dtype=torch.int32, device=dev)
    d = torch.empty((px, px), dtype=torch.float64, device=dev)
    wsd = cc.workspace(cc.cc_distance_map_workspace_bytes(px, px), dev)
    stream = torch.cuda.current_stream(dev)
    res = None
    for it in range(2):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        fld = cc.cc_field_create(xs, ys, mm, f.kappa_s, f.gamma, fopt)
        cc.cc_critical_curves(fld, m, z, w, None, ws, stream)
        ev[1].record(stream)
        cc.cc_crossing_map(w, -ext, ext, -ext, ext, px, px, ncc, stream)
        ev[2].record(stream)
        cc.cc_distance_map(ncc, 2 * ext / px, d, wsd, stream)
        ev[3].record(stream)
        ev[3].synchronize()
        st, rep = cc.cc_field_report(fld)
        res = (ev, st, rep)
        del fld
    ev, st, rep = res
    total = ev[0].elapsed_time(ev[3])
    roots = (m + 1) * nr
    del z, w, ncc, d, ws, wsd
    torch.cuda.empty_cache()
    return {"value": round(roots / (total / 1e3), 1), "unit": UNIT, "ms": round(total, 1), "steps": 1, "warmup": 1,
            "roots": roots, "stages_ms": {"trace": round(rep["trace_ms"], 2), "join": round(rep["join_ms"], 2),
                                          "polish_caustic": round(rep["polish_ms"], 2),
                                          "crossing": round(ev[1].elapsed_time(ev[2]), 2),
                                          "distance": round(ev[2].elapsed_time(ev[3]), 2)},
            "status_ok": st == cc.CC_OK, "max_err_est": rep["max_err_est"], "uncertified": rep["uncertified"],
            "subchains": rep["subchains"],
            "workload": f"N=20000 Kroupa-like, kappa_*=0.2, kappa_s=0.3, gamma=0.3, m={m}, {px}^2 maps over +-{ext}"}


def _match_rows(zg, zo):
    """Nearest-neighbour pairing of the GPU's points to the oracle's (one row each): index
    into zo per GPU point and the pairing distance."""
    from scipy.spatial import cKDTree
    d, idx = cKDTree(np.stack([zo.real, zo.imag], axis=1)).query(np.stack([zg.real, zg.imag], axis=1))
    return idx, d


def cpu_baseline(f, m, ext, px, seconds, host):
    """The FP64 oracle on this host's cores, on a bounded sample of the same step, scaled
    to the whole step (a1-a7):
      - warm-started rows after the centre row (Aberth + Newton polish + caustic mapping),
        time per row x (m + 1) rows;
      - whole pixel rows of the crossing map over all of the GPU step's caustic segments,
        time per pixel row x the map's rows;
      - the distance map of the GPU step's N_cc map, whole.
    The same legs once more on one thread (fewer rows).  Also returns the FP64-oracle error
    of the GPU step's results: the Newton correction and lens map of every point, the points
    of the oracle's solved rows, and crossing-map and distance-map mismatches."""
    import oracle
    nr = 2 * f.n
    roots = (m + 1) * nr
    pixel = 2 * ext / px
    cores = oracle.num_threads()
    c = m // 2
    z, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(c, m))  # untimed seed
    seed = z.copy()
    solved = {}
    t0 = time.perf_counter()
    while True:
        j = c + 1 + len(solved)
        z, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, m), z0=z)
        solved[j] = (z, oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, z))
        if time.perf_counter() - t0 > 0.5 * seconds or len(solved) >= 200:
            break
    t_row = (time.perf_counter() - t0) / len(solved)
    u = np.arange(16) + 0.5
    prow = sorted({int(v * px / 16) for v in u})
    t0 = time.perf_counter()
    ref_rows = oracle.crossing_rows(host["w"], -ext, ext, -ext, ext, px, px, prow)
    t_cross = (time.perf_counter() - t0) * px / len(prow)
    t0 = time.perf_counter()
    ref_d = oracle.distance_map(host["ncc"], pixel)
    t_dist = time.perf_counter() - t0
    step_s = t_row * (m + 1) + t_cross + t_dist

    # one thread: 4 rows, one pixel row, the distance map
    oracle.set_num_threads(1)
    try:
        zz = seed
        t0 = time.perf_counter()
        for k in range(4):
            zz, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(c + 1 + k, m), z0=zz)
            oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zz)
        t_row1 = (time.perf_counter() - t0) / 4
        t0 = time.perf_counter()
        oracle.crossing_rows(host["w"], -ext, ext, -ext, ext, px, px, [px // 2])
        t_cross1 = (time.perf_counter() - t0) * px
        t0 = time.perf_counter()
        oracle.distance_map(host["ncc"], pixel)
        t_dist1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    step1_s = t_row1 * (m + 1) + t_cross1 + t_dist1

    # FP64-oracle error of the GPU step's results
    step, wo = oracle.newton_check(f.x, f.y, f.m, f.kappa_s, f.gamma, m, host["z"])
    dz_rows = dw_rows = 0.0
    for j, (zo, wjo) in solved.items():
        idx, d = _match_rows(host["z"][j], zo)
        dz_rows = max(dz_rows, float(d.max()))
        dw_rows = max(dw_rows, float(np.abs(host["w"][j] - wjo[idx]).max()))
    ncc_bad = int((host["ncc"][prow] != ref_rows).sum())
    d_bad = int((host["d"] != ref_d).sum())
    accuracy = {"points_checked": int(step.size), "max_newton_step": float(step.max()),
                "points_newton_step_ge_1e-9": int((step >= 1e-9).sum()),
                "max_abs_w_minus_oracle_w_at_gpu_z": float(np.abs(host["w"] - wo).max()),
                "oracle_rows": len(solved), "max_abs_dz_oracle_rows": dz_rows, "max_abs_dw_oracle_rows": dw_rows,
                "ncc_pixels_checked": len(prow) * px, "ncc_mismatches": ncc_bad,
                "distance_pixels_checked": int(ref_d.size), "distance_mismatches": d_bad,
                "note": "every point: FP64 Newton correction |F/F'| and oracle w at the GPU's z; the oracle's own "
                        "warm-started rows matched point by point; whole crossing-map rows and the whole "
                        "distance map (from the GPU's N_cc) compared exactly"}
    return {"value": round(roots / step_s, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(solved)} warm-started rows (Aberth + Newton polish + caustics) x (m+1)/{len(solved)}, "
                      f"{len(prow)} whole pixel rows of the {px}^2 crossing map over all caustic segments x "
                      f"{px}/{len(prow)}, the whole {px}^2 distance map; {cores} threads",
            "step_s": round(step_s, 2),
            "legs_s": {"rows": round(t_row * (m + 1), 2), "crossing_map": round(t_cross, 2),
                       "distance_map": round(t_dist, 2)},
            "one_thread": {"value": round(roots / step1_s, 1), "cores": 1, "step_s": round(step1_s, 2),
                           "legs_s": {"rows": round(t_row1 * (m + 1), 2), "crossing_map": round(t_cross1, 2),
                                      "distance_map": round(t_dist1, 2)},
                           "sample": "4 warm rows, 1 pixel row of the crossing map, the whole distance map"},
            "accuracy": accuracy}


def run_reference(args):
    """Reference arm: the FP64 oracle (the only reference implementation of this method)
    timed as it stands on the host cores.  Each step is a bounded sample of the whole
    step, scaled to it: R warm-started rows (Aberth + Newton polish + caustics) x (m+1)/R,
    the crossing map of those rows' caustic segments over every pixel row x m/R, and the
    distance map of that crossing map."""
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import oracle
    wl = workload(args.workload, args.msteps, args.map)
    f = wl.fields[0]
    m = wl.msteps
    ext, px = wl.map_extent, wl.map_pixels
    nr = 2 * f.n
    c = m // 2
    z, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(c, m))
    w = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, z)
    R = 20
    times, legs = [], []
    j = c
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        zs, ws_ = [z], [w]
        for _ in range(R):
            j += 1
            z, _ = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, m), z0=z)
            w = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, z)
            zs.append(z)
            ws_.append(w)
        t1 = time.perf_counter()
        ncc = oracle.crossing_map(np.array(ws_), -ext, ext, -ext, ext, px, px)
        t2 = time.perf_counter()
        oracle.distance_map(ncc, 2 * ext / px)
        t3 = time.perf_counter()
        if k >= args.warmup:
            leg = ((t1 - t0) * (m + 1) / R, (t2 - t1) * m / R, t3 - t2)
            legs.append(leg)
            times.append(sum(leg))
    step_s = sum(times) / len(times)
    value = (m + 1) * nr / step_s
    sample = (f"per step: {R} warm-started rows of the {f.n}-star, m={m} field (Aberth + Newton polish + caustics) "
              f"x (m+1)/{R}, the {px}^2 crossing map of their caustic segments x m/{R}, and its distance map; "
              f"FP64 oracle")
    out = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * step_s, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl.name, "n_stars": f.n, "n_roots": nr, "phi_steps": m},
           "impl": "reference",
           "legs_s": {"rows": round(statistics.mean(l[0] for l in legs), 2),
                      "crossing_map": round(statistics.mean(l[1] for l in legs), 2),
                      "distance_map": round(statistics.mean(l[2] for l in legs), 3)},
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
