"""The request server on the GPU: requests that overlap on the device give the same
results as each request run alone (bit for bit: a request's kernels and shapes do not
depend on what else is in flight), a repeated field reuses its resident caustics, and a
degenerate request fails alone without disturbing the others."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import cc, synth
from paper_2506_02121_gb300.serve import GpuExecutor, Request, Server, summarize
from tests.gpu_util import compare_chain

pytestmark = pytest.mark.gpu


def _requests():
    reqs = []
    for i, n in enumerate([40, 160, 12, 300, 75, 220]):
        u = synth.uniform(synth.stream_seed(6, i, 2), 2)
        f = synth.disc_field(n, 0.1 + 0.6 * u[0], 0.0, 0.8 * u[1], synth.stream_seed(6, i), "loguniform")
        reqs.append(Request(rid=i, arrival=0.002 * i, x=f.x, y=f.y, mass=f.m, kappa_s=0.0, gamma=f.gamma,
                            msteps=60, map_extent=6.0, map_pixels=128, field_key=f"field{i}"))
    # the same field again (resident caustics reused) and a degenerate macro-model
    r0 = reqs[0]
    reqs.append(Request(rid=6, arrival=0.5, x=r0.x, y=r0.y, mass=r0.mass, kappa_s=0.0, gamma=r0.gamma,
                        msteps=60, map_extent=6.0, map_pixels=128, field_key="field0"))
    reqs.append(Request(rid=7, arrival=0.003, x=r0.x, y=r0.y, mass=r0.mass, kappa_s=0.2, gamma=0.8,
                        msteps=60, map_extent=6.0, map_pixels=128))
    return reqs


def test_mix_equals_alone_and_reuse():
    reqs = _requests()
    srv = Server(GpuExecutor(slots=3), slots=3, budget_bytes=8 << 30)
    mixed = {r.rid: r for r in srv.run(reqs, realtime=True)}
    st = summarize(list(mixed.values()), wall=max(r.finished for r in mixed.values() if r.status == "ok"))
    assert mixed[7].status == "error"
    assert all(mixed[i].status == "ok" for i in range(7)), [(r.rid, r.status, r.error) for r in mixed.values()]
    assert mixed[6].reused and not mixed[0].reused
    assert torch.equal(mixed[6].outputs["ncc"], mixed[0].outputs["ncc"])
    assert st["p50_s"] is not None and st["p99_s"] >= st["p50_s"]
    for i in range(6):
        alone = Server(GpuExecutor(slots=1), slots=1, budget_bytes=8 << 30).run([reqs[i]], realtime=False)[0]
        assert alone.status == "ok"
        for k in ("z", "w", "ncc"):
            assert torch.equal(alone.outputs[k], mixed[i].outputs[k]), (i, k)
    # and the served result is right
    r = reqs[3]
    zo, _, _ = oracle.critical_curves(np.asarray(r.x), np.asarray(r.y), np.asarray(r.mass), r.kappa_s, r.gamma,
                                      r.msteps)
    compare_chain(mixed[3].outputs["z"].cpu().numpy(), zo, 1e-9)


def test_served_size_request_alone_equals_mix_and_oracle():
    """A request of the served workload's largest size (N = 19405 stars, log-uniform masses,
    m = 200, a 1024^2 map over +-10; the cluster tracer runs it) beside three smaller ones
    from the same trace: bit-identical alone and in the mix, and its sampled rows pass the
    oracle's FP64 Newton check (every point of each row within 1e-9 of a distinct zero of F,
    caustics within 1e-9 of the oracle's lens map)."""
    from scipy.spatial import cKDTree
    trace = synth.served_requests(69, 50.0)
    pick = [68, 3, 10, 25]
    reqs = []
    for k, i in enumerate(pick):
        t, f = trace[i]
        reqs.append(Request(rid=k, arrival=0.001 * k, x=f.x, y=f.y, mass=f.m, kappa_s=f.kappa_s, gamma=f.gamma,
                            msteps=200, map_extent=10.0, map_pixels=1024))
    assert reqs[0].n == 19405
    mixed = {r.rid: r for r in Server(GpuExecutor(slots=4), slots=4, budget_bytes=32 << 30).run(reqs, realtime=True)}
    assert all(r.status == "ok" for r in mixed.values()), [(r.rid, r.status, r.error) for r in mixed.values()]
    alone = Server(GpuExecutor(slots=1), slots=1, budget_bytes=32 << 30).run([reqs[0]], realtime=False)[0]
    assert alone.status == "ok"
    for k in ("z", "w", "ncc"):
        assert torch.equal(alone.outputs[k], mixed[0].outputs[k]), k
    r = reqs[0]
    z = mixed[0].outputs["z"]
    w = mixed[0].outputs["w"]
    rows = [0, 57, 100, 143, 200]
    zs = z[rows].cpu().numpy()
    ws = w[rows].cpu().numpy()
    for t, j in enumerate(rows):
        step, wo = oracle.newton_check(np.asarray(r.x), np.asarray(r.y), np.asarray(r.mass), r.kappa_s, r.gamma,
                                       r.msteps, zs[t:t + 1], row0=j)
        assert step.max() < 1e-9, (j, float(step.max()))
        assert np.abs(ws[t] - wo[0]).max() < 1e-9, j
        pts = np.stack([zs[t].real, zs[t].imag], axis=1)
        d, nb = cKDTree(pts).query(pts, k=2)
        assert (d[:, 1] > 2e-9 + step[0] + step[0][nb[:, 1]]).all(), f"row {j}: two points share a zero"
