"""Host-side logic of the request server, on the CPU with a fake executor: FIFO admission
under slots and an HBM budget, overlap of in-flight requests, oversized and failing
requests reported without stopping the server, and latency percentiles."""
import pytest

from paper_2506_02121_gb300.serve import AdmissionPolicy, Request, Server, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    """Each request 'runs' for n / 100 time units after admission; rid 13 fails."""

    def __init__(self, clock):
        self.clock = clock
        self.max_inflight = 0
        self.inflight = 0
        self.order = []

    def estimate_bytes(self, req):
        return req.n * 10

    def start(self, req, slot):
        self.inflight += 1
        self.max_inflight = max(self.max_inflight, self.inflight)
        self.order.append(req.rid)
        return {"req": req, "end": self.clock.t + req.n / 100.0}

    def done(self, h):
        return self.clock.t >= h["end"]

    def finish(self, h):
        self.inflight -= 1
        if h["req"].rid == 13:
            raise RuntimeError("injected failure")
        return "ok", "", 2 * h["req"].n * (h["req"].msteps + 1), False, None


def _requests():
    out = []
    for i in range(20):
        n = 50 + 37 * (i % 7)
        out.append(Request(rid=i, arrival=0.05 * i, x=[0.0] * n, y=[0.0] * n, mass=[1.0] * n,
                           kappa_s=0.0, gamma=0.3, msteps=10))
    out.append(Request(rid=99, arrival=0.2, x=[0.0] * 5000, y=[0.0] * 5000, mass=[1.0] * 5000,
                       kappa_s=0.0, gamma=0.3))  # larger than the budget
    return out


def _drive(server, clock, reqs, step=0.01):
    pending = sorted(reqs, key=lambda r: r.arrival)
    i = 0
    while i < len(pending) or not server.idle():
        while i < len(pending) and pending[i].arrival <= clock.t:
            server.submit(pending[i])
            i += 1
        server.poll()
        clock.t += step
        assert server.policy.used <= server.policy.budget
        assert len(server.running) <= server.policy.slots


def test_admission_fifo_budget_and_overlap():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    srv = Server(ex, slots=3, budget_bytes=9000, clock=clock)
    reqs = _requests()
    _drive(srv, clock, reqs)
    res = {r.rid: srv.results[r.rid] for r in reqs}
    assert res[99].status == "error" and "budget" in res[99].error
    assert res[13].status == "error" and "injected" in res[13].error
    assert all(res[i].status == "ok" for i in range(20) if i != 13)
    assert ex.order == sorted(ex.order)          # first come, first served
    assert ex.max_inflight >= 2                  # requests overlap
    for r in res.values():
        if r.status == "ok":
            assert r.admitted >= r.arrival - 1e-9 and r.finished >= r.admitted
    st = summarize(list(res.values()), wall=clock.t)
    assert st["ok"] == 19 and st["errors"] == 2
    assert st["p50_s"] <= st["p99_s"]


def test_policy_never_overtakes_a_blocked_head():
    p = AdmissionPolicy(slots=4, budget_bytes=100)
    p.push("big", 80)
    p.push("small", 10)
    assert p.pop_admissible() == ("big", 80)
    p.push("big2", 50)
    p.push("tiny", 1)
    assert p.pop_admissible() == ("small", 10)
    assert p.pop_admissible() is None            # big2 does not fit; tiny waits behind it
    p.release(80)
    assert p.pop_admissible() == ("big2", 50)
    assert p.pop_admissible() == ("tiny", 1)
    with pytest.raises(ValueError):
        AdmissionPolicy(0, 10)


class TickClock:
    """Advances by a fixed step at every reading (the server loop reads it as it polls)."""

    def __init__(self, step=1e-3):
        self.t = 0.0
        self.step = step

    def __call__(self):
        self.t += self.step
        return self.t


def test_all_at_once_latency_runs_from_submission():
    """Requests fed all at once ahead of their arrival times: latency counts from the
    submission (never negative); fed in real time it counts from the arrival."""
    for realtime in (False, True):
        clock = TickClock()
        ex = FakeExecutor(clock)
        srv = Server(ex, slots=3, budget_bytes=9000, clock=clock)
        reqs = [r for r in _requests() if r.rid not in (13, 99)]
        res = srv.run(reqs, realtime=realtime, sleep=0)
        assert all(r.status == "ok" for r in res)
        assert all(r.latency >= 0.0 for r in res)
        if not realtime:
            assert max(r.arrival for r in res) < 0.05   # every request submitted at the start
        else:
            assert [r.arrival for r in res] == [q.arrival for q in reqs]
