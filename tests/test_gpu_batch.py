"""Batched launches (many fields of uneven N in one persistent launch): every field matches
the FP64 oracle within 1e-9, graph replay reproduces a direct launch bit for bit, and the
autotuner returns one of its candidates and caches it."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import autotune, cc, synth
from tests.gpu_util import compare_chain

pytestmark = pytest.mark.gpu


def _fields():
    spec = [(1, 40), (3, 22), (7, 60), (20, 120), (50, 48), (120, 30), (200, 16), (33, 300), (2, 10), (90, 64)]
    out = []
    for i, (n, m) in enumerate(spec):
        u = synth.uniform(synth.stream_seed(5, i, 3), 3)
        ks, g, kst = 0.25 * u[0], 0.7 * u[1], 0.1 + 0.6 * u[2]
        if abs(1 - ks - g) < 0.01:
            g += 0.05
        f = synth.disc_field(n, kst, ks, g, synth.stream_seed(5, i), "unit" if i % 2 else "loguniform")
        out.append((f, m))
    return out


@pytest.fixture(scope="module")
def batch_run():
    spec = _fields()
    fields = [cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma) for f, _ in spec]
    ms = [m for _, m in spec]
    b = cc.batch_critical_curves(fields, ms, caustics=True)
    st, per, tot = cc.cc_batch_report(b)
    return spec, fields, ms, b, st, per, tot


def test_batch_matches_oracle_per_field(batch_run):
    spec, fields, ms, b, st, per, tot = batch_run
    assert st == cc.CC_OK, tot
    for (f, m), z, w in zip(spec, b.z, b.w):
        zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, m)
        assert bad == 0
        zg = z.cpu().numpy()
        worst, pairs = compare_chain(zg, zo, 1e-9)
        wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zo)
        wg = w.cpu().numpy()
        for j, idx in enumerate(pairs):
            assert np.abs(wg[j] - wo[j][idx]).max() < 1e-9
    assert tot["unconverged"] == 0 and tot["uncertified"] == 0 and tot["seam_ambiguous"] == 0
    info = cc.cc_batch_info(b)
    assert info["items"] >= len(spec)


def test_graph_replay_equals_direct_launch(batch_run):
    spec, fields, ms, b, st, per, tot = batch_run
    ref = [z.clone() for z in b.z]
    refw = [w.clone() for w in b.w]
    s = torch.cuda.Stream()
    for _ in range(2):
        for z in b.z:
            z.zero_()
        cc.cc_batch_launch(b, True, s)
        s.synchronize()
        assert all(torch.equal(a, c) for a, c in zip(b.z, ref))
        assert all(torch.equal(a, c) for a, c in zip(b.w, refw))
    st2, _, tot2 = cc.cc_batch_report(b)
    assert st2 == cc.CC_OK


def test_batched_field_equals_single_field_solve(batch_run):
    spec, fields, ms, b, st, per, tot = batch_run
    k = 7  # N = 33, m = 300
    z1, _, _ = cc.critical_curves(fields[k], ms[k], caustics=False)
    compare_chain(b.z[k].cpu().numpy(), z1.cpu().numpy(), 1e-9)


def test_autotuner_picks_a_candidate_and_caches(tmp_path, batch_run):
    spec, fields, ms, b, st, per, tot = batch_run
    path = str(tmp_path / "tune.json")
    t, i, info = autotune.tune(fields, ms, probe_steps=16, repeats=1, cache_path=path)
    assert (t, i) in autotune.CANDIDATES and not info["cached"]
    t2, i2, info2 = autotune.tune(fields, ms, cache_path=path)
    assert (t2, i2) == (t, i) and info2["cached"]
    b2 = cc.batch_critical_curves(fields[:3], ms[:3], caustics=False, block_threads=t, items_per_cta=i)
    assert cc.cc_batch_report(b2)[0] == cc.CC_OK
