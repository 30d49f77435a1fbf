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
