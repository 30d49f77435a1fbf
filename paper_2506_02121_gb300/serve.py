"""Continuous-batching request server for critical-curve / caustic / crossing-map requests.

Requests (a star field, its macro-model, m phi steps and a source-plane map) arrive at
arbitrary times.  The server admits them as execution slots and device memory free up,
first come first served, and runs every admitted request on its own CUDA stream.  Work of
different requests therefore overlaps on the GPU: one request's polish blocks fill SMs
while another's tracing CTAs still run.  A request only queues while no slot is free or
its memory does not fit the HBM budget.

Fields stay resident on the device (their star arrays as cc_field handles, and the traced
chain matrix and caustics of the last m), keyed by a caller-chosen field key, within the
same HBM budget (least recently used entries are evicted first).  A repeated request for
a resident field and m reuses the traced caustics and only rasterises its map.

Latency is measured from arrival to the completion event of the request's last kernel;
p50/p99 are reported beside roots/s.  Results do not depend on what else is in flight:
a request's kernels, sub-range count and block size depend only on the request itself.

The admission policy (AdmissionPolicy) is plain Python with no GPU dependency, so its
logic is tested on the CPU with a fake executor.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time
from typing import Any, Callable, Optional


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds on the server clock
    x: Any
    y: Any
    mass: Any
    kappa_s: float
    gamma: float
    msteps: int = 200
    map_extent: float = 10.0
    map_pixels: int = 1024
    field_key: Optional[str] = None  # requests sharing a key reuse the resident field

    @property
    def n(self) -> int:
        return len(self.x)


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float = math.nan
    finished: float = math.nan
    status: str = "pending"      # ok | noconv | error
    error: str = ""
    roots: int = 0
    reused: bool = False
    outputs: Any = None          # executor-specific (device tensors)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class AdmissionPolicy:
    """FIFO admission under a slot count and a device-memory budget (bytes)."""

    def __init__(self, slots: int, budget_bytes: int):
        if slots < 1 or budget_bytes <= 0:
            raise ValueError("need slots >= 1 and a positive budget")
        self.slots = slots
        self.budget = int(budget_bytes)
        self.used = 0
        self.inflight = 0
        self.queue: collections.deque = collections.deque()

    def push(self, item, nbytes: int):
        self.queue.append((item, int(nbytes)))

    def fits_ever(self, nbytes: int) -> bool:
        return nbytes <= self.budget

    def pop_admissible(self):
        """Next request that may start now (head of the queue only: no overtaking), or None."""
        if not self.queue or self.inflight >= self.slots:
            return None
        item, nb = self.queue[0]
        if self.used + nb > self.budget:
            return None
        self.queue.popleft()
        self.used += nb
        self.inflight += 1
        return item, nb

    def release(self, nbytes: int):
        self.used -= int(nbytes)
        self.inflight -= 1
        assert self.used >= 0 and self.inflight >= 0


class Server:
    """Drives an executor with the admission policy.

    executor must provide:
      estimate_bytes(request) -> int         device bytes the request holds while in flight
      start(request, slot) -> handle         enqueue the request's work (non-blocking)
      done(handle) -> bool                   completion test (non-blocking)
      finish(handle) -> (status, error, roots, reused, outputs)
    """

    def __init__(self, executor, slots: int = 4, budget_bytes: int = 64 << 30,
                 clock: Callable[[], float] = time.perf_counter):
        self.ex = executor
        self.policy = AdmissionPolicy(slots, budget_bytes)
        self.clock = clock
        self.t0 = clock()
        self.realtime = True
        self.results: dict = {}
        self.running: dict = {}   # slot -> (request, handle, nbytes)
        self.free_slots = list(range(slots))

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request):
        # latency runs from the arrival, or from the submission when requests are fed all at
        # once ahead of their arrival times
        res = Result(req.rid, req.arrival if self.realtime else self.now())
        self.results[req.rid] = res
        nb = self.ex.estimate_bytes(req)
        if not self.policy.fits_ever(nb):
            res.status, res.error, res.finished = "error", f"request needs {nb} B > budget", self.now()
            return
        self.policy.push(req, nb)

    def poll(self):
        """Retire finished requests, then admit as many queued ones as fit."""
        for slot in list(self.running):
            req, h, nb = self.running[slot]
            if self.ex.done(h):
                res = self.results[req.rid]
                try:
                    res.status, res.error, res.roots, res.reused, res.outputs = self.ex.finish(h)
                except Exception as e:  # a failing request never takes the server down
                    res.status, res.error = "error", f"{type(e).__name__}: {e}"
                res.finished = self.now()
                del self.running[slot]
                self.free_slots.append(slot)
                self.policy.release(nb)
        while True:
            nxt = self.policy.pop_admissible()
            if nxt is None:
                break
            req, nb = nxt
            slot = self.free_slots.pop()
            res = self.results[req.rid]
            res.admitted = self.now()
            try:
                h = self.ex.start(req, slot)
            except Exception as e:
                res.status, res.error, res.finished = "error", f"{type(e).__name__}: {e}", self.now()
                self.free_slots.append(slot)
                self.policy.release(nb)
                continue
            self.running[slot] = (req, h, nb)

    def idle(self) -> bool:
        return not self.running and not self.policy.queue

    def run(self, requests, realtime: bool = True, sleep: float = 2e-4):
        """Feed requests at their arrival times (realtime) or all at once; return results."""
        pending = sorted(requests, key=lambda r: r.arrival)
        i = 0
        self.realtime = realtime
        self.t0 = self.clock()
        while i < len(pending) or not self.idle():
            t = self.now()
            while i < len(pending) and (not realtime or pending[i].arrival <= t):
                self.submit(pending[i])
                i += 1
            self.poll()
            if realtime and i < len(pending) and self.idle():
                wait = pending[i].arrival - self.now()
                if wait > 0:
                    time.sleep(min(wait, 0.01))
            elif sleep:
                time.sleep(sleep)
        return [self.results[r.rid] for r in requests]


def summarize(results, wall: float):
    ok = [r for r in results if r.status == "ok"]
    lat = sorted(r.latency for r in ok)

    def pct(p):
        if not lat:
            return None
        k = min(len(lat) - 1, max(0, int(math.ceil(p / 100.0 * len(lat))) - 1))
        return lat[k]

    roots = sum(r.roots for r in ok)
    return {"requests": len(results), "ok": len(ok), "errors": sum(r.status == "error" for r in results),
            "noconv": sum(r.status == "noconv" for r in results), "reused": sum(r.reused for r in ok),
            "p50_s": pct(50), "p99_s": pct(99), "mean_s": (sum(lat) / len(lat)) if lat else None,
            "roots": roots, "wall_s": wall, "roots_per_s": roots / wall if wall > 0 else None}


class GpuExecutor:
    """Runs requests through the C ABI on one CUDA stream per slot.

    precision selects the solver form: "mixed" (FP32 Aberth tracer + certified polish, the
    library default) or "fp64" (the paper's plain FP64 Aberth form with FP64 caustics), so
    that one request trace can be served by both."""

    def __init__(self, slots: int, block_threads: int = 0, subchains: int = 0, device: int = 0,
                 cache_bytes: int = 8 << 30, precision: str = "mixed"):
        import torch

        from . import cc
        self.torch = torch
        self.cc = cc
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]
        self.block_threads = block_threads
        self.subchains = subchains
        self.cache = collections.OrderedDict()  # key -> (field, m, z, w, bytes)
        self.cache_bytes = cache_bytes
        self.cache_used = 0
        if precision not in ("mixed", "fp64"):
            raise ValueError("precision must be 'mixed' or 'fp64'")
        self.precision = precision

    def _opts(self):
        o = self.cc.cc_options_default()
        o.block_threads = self.block_threads
        o.subchains = self.subchains
        if self.precision == "fp64":
            o.precision = self.cc.CC_FP64
            o.hp_arith = self.cc.CC_HP_FP64
        return o

    def estimate_bytes(self, req: Request) -> int:
        rows, nr = req.msteps + 1, 2 * req.n
        zw = 2 * 16 * rows * nr
        # tracer rows (complex64, or complex128 in the FP64 form) + iteration counts, plus
        # joins and per-CTA Jacobi state for at most 320 sub-ranges (about 100 bytes per
        # root each)
        ws = rows * nr * ((16 if self.precision == "fp64" else 8) + 4) + 320 * 100 * nr
        return zw + ws + 4 * req.map_pixels ** 2

    def start(self, req: Request, slot: int):
        torch, cc = self.torch, self.cc
        s = self.streams[slot]
        key = req.field_key
        hit = self.cache.get(key) if key is not None else None
        with torch.cuda.stream(s):
            if hit is not None and hit[1] == req.msteps:
                self.cache.move_to_end(key)
                field, _, z, w, _ = hit
                reused = True
                ws = None
            else:
                field = cc.cc_field_create(req.x, req.y, req.mass, req.kappa_s, req.gamma, self._opts())
                rows = req.msteps + 1
                z = torch.empty((rows, field.n_roots), dtype=torch.complex128, device=self.dev)
                w = torch.empty_like(z)
                ws = cc.workspace(cc.cc_critical_curves_workspace_bytes(field, req.msteps), self.dev)
                cc.cc_critical_curves(field, req.msteps, z, w, None, ws, s)
                reused = False
            e = req.map_extent
            ncc = torch.empty((req.map_pixels, req.map_pixels), dtype=torch.int32, device=self.dev)
            cc.cc_crossing_map(w, -e, e, -e, e, req.map_pixels, req.map_pixels, ncc, s)
            ev = torch.cuda.Event()
            ev.record(s)
        return {"req": req, "field": field, "z": z, "w": w, "ncc": ncc, "ws": ws, "ev": ev, "reused": reused}

    def done(self, h) -> bool:
        return h["ev"].query()

    def finish(self, h):
        cc = self.cc
        req = h["req"]
        status, err = "ok", ""
        if not h["reused"]:
            st, rep = cc.cc_field_report(h["field"])
            if st != cc.CC_OK:
                status, err = "noconv", f"unconverged={rep['unconverged']} uncertified={rep['uncertified']}"
            if req.field_key is not None:
                nb = 2 * h["z"].numel() * 16
                self.cache[req.field_key] = (h["field"], req.msteps, h["z"], h["w"], nb)
                self.cache_used += nb
                while self.cache_used > self.cache_bytes and len(self.cache) > 1:
                    _, old = self.cache.popitem(last=False)
                    self.cache_used -= old[4]
        h["ws"] = None
        return status, err, h["z"].numel(), h["reused"], {"z": h["z"], "w": h["w"], "ncc": h["ncc"]}
