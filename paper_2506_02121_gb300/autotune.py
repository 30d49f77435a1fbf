"""Autotuner for the batched launch's tile shape.

The batched tracer has two shape knobs: the CTA size of the persistent tracing launch
(threads per block, which with the kernel's registers fixes how many CTAs stay resident per
SM) and how finely the fields are cut into (field, phi sub-range) work items per resident
CTA (finer items balance better, but every item pays a cold Aberth start).  The tuner times
each candidate on a short probe of the same fields (same stars, fewer phi steps) with CUDA
events, picks the fastest, and caches the choice in a JSON file keyed by the batch's
N distribution (log2 buckets), phi-step bucket and the GPU name.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import cc

CANDIDATES = [(512, 4), (512, 8), (256, 4), (256, 8), (128, 8)]


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "ccgpu", "autotune.json")


def shape_key(fields, msteps) -> str:
    hist = {}
    for f in fields:
        b = int(math.log2(max(f.n, 1)))
        hist[b] = hist.get(b, 0) + 1
    mb = int(math.log2(max(1, int(sum(msteps) / len(msteps)))))
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    h = ",".join(f"{k}:{hist[k]}" for k in sorted(hist))
    return f"{name}|N[{h}]|m2^{mb}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _time_candidate(fields, probe_m, threads, items, repeats):
    b = cc.cc_batch_create(fields, probe_m, threads, items)
    z = [torch.empty((m + 1, f.n_roots), dtype=torch.complex128, device="cuda") for f, m in zip(fields, probe_m)]
    ws = cc.workspace(cc.cc_batch_workspace_bytes(b))
    cc.cc_batch_bind(b, z, None, ws)
    stream = torch.cuda.current_stream()
    cc.cc_batch_launch(b, False, stream)  # warm-up
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cc.cc_batch_launch(b, False, stream)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    cc.cc_batch_destroy(b)
    return best


def tune(fields, msteps, probe_steps: int = 64, repeats: int = 2, cache_path: str | None = None,
         candidates=CANDIDATES, refresh: bool = False):
    """Returns (block_threads, items_per_cta, info) for this batch, from the cache when present."""
    path = cache_path or default_cache_path()
    key = shape_key(fields, msteps)
    cache = _load(path)
    if not refresh and key in cache:
        e = cache[key]
        return e["block_threads"], e["items_per_cta"], {"cached": True, "key": key}
    probe_m = [max(2, min(int(m), probe_steps) // 2 * 2) for m in msteps]
    timings = {}
    for threads, items in candidates:
        timings[f"{threads}x{items}"] = _time_candidate(fields, probe_m, threads, items, repeats)
    best = min(timings, key=timings.get)
    threads, items = (int(v) for v in best.split("x"))
    cache[key] = {"block_threads": threads, "items_per_cta": items, "probe_ms": timings}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return threads, items, {"cached": False, "key": key, "probe_ms": timings}
