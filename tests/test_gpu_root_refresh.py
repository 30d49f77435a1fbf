"""The near/far split of the FP32 tracer's Aberth root sum (root_refresh = K >= 2): the
roots and caustics are the same zeros of F as with the exact sum in every sweep (within
1e-9 of the oracle, row by row), on fields whose sub-ranges take both the blocked sweep and
the few-roots path, the disc and the rectangle, single and batched; fewer root terms are
summed; and the result does not depend on the launch (graph replay equals a direct launch)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import cc, synth
from tests.gpu_util import compare_chain

pytestmark = pytest.mark.gpu


def _opt(k, base=None):
    # few sub-ranges, so that warm rows (where the split applies) dominate the work
    o = cc.cc_options_default() if base is None else base
    o.root_refresh = k
    o.subchains = 4
    return o


# (400, 1024, 64): the library's default refresh period with 256 rows per sub-range, so
# every sub-range crosses three refreshes
@pytest.mark.parametrize("n,m,k", [(300, 400, 8), (500, 300, 4), (40, 300, 16), (800, 160, 2), (400, 1024, 64)])
def test_split_matches_oracle_and_exact_sum(n, m, k):
    f = synth.disc_field(n, 0.45, 0.05, 0.35, synth.stream_seed(11, n), "loguniform", 0.08, 1.0)
    zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, m)
    assert bad == 0
    out = {}
    for kk in (0, k):
        fld = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, _opt(kk))
        z, w, _ = cc.critical_curves(fld, m, caustics=True)
        st, rep = cc.cc_field_report(fld)
        assert st == cc.CC_OK, rep
        assert rep["unconverged"] == 0 and rep["uncertified"] == 0 and rep["seam_ambiguous"] == 0
        worst, pairs = compare_chain(z.cpu().numpy(), zo, 1e-9)
        wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zo)
        wg = w.cpu().numpy()
        for j, idx in enumerate(pairs):
            assert np.abs(wg[j] - wo[j][idx]).max() < 1e-9
        out[kk] = rep
    nr = 2 * n
    assert out[0]["root_terms"] == out[0]["root_iterations"] * nr
    assert out[k]["root_terms"] < 0.75 * out[0]["root_terms"]
    assert out[k]["jumped"] == 0


def test_split_rectangle():
    n, m = 200, 100
    f = synth.rect_field(n, 0.3, 0.1, 0.3, synth.stream_seed(12, 0), 0.7, "loguniform")
    t = oracle.rect_choose_t(f.kappa_star, f.c1, f.c2)
    fld = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, _opt(8, cc.rect_options(f.kappa_star, f.c1, f.c2)))
    assert fld.n_roots == 2 * n + t - 1
    z, w, _ = cc.critical_curves(fld, m, caustics=True)
    st, rep = cc.cc_field_report(fld)
    assert st == cc.CC_OK, rep
    R = oracle.Rect(f.kappa_star, f.c1, f.c2, t)
    zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, m, rect=R)
    assert bad == 0
    worst, pairs = compare_chain(z.cpu().numpy(), zo, 1e-9)
    wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zo, rect=R)
    wg = w.cpu().numpy()
    for j, idx in enumerate(pairs):
        assert np.abs(wg[j] - wo[j][idx]).max() < 1e-9


def test_split_batched_equals_single_and_replay():
    spec = [(150, 200), (600, 120), (35, 300), (900, 80)]
    fields, ms, flds = [], [], []
    for i, (n, m) in enumerate(spec):
        f = synth.disc_field(n, 0.2 + 0.1 * i, 0.1, 0.3, synth.stream_seed(13, i))
        flds.append(f)
        fields.append(cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, _opt(8)))
        ms.append(m)
    b = cc.batch_critical_curves(fields, ms, caustics=True)
    st, per, tot = cc.cc_batch_report(b)
    assert st == cc.CC_OK, tot
    ref = [z.clone() for z in b.z]
    s = torch.cuda.Stream()
    cc.cc_batch_launch(b, True, s)
    s.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(b.z, ref))
    for f, m, z in zip(flds, ms, b.z):
        zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, m)
        compare_chain(z.cpu().numpy(), zo, 1e-9)


@pytest.mark.parametrize("k", [0, 8])
def test_repeated_solves_are_bit_identical(k):
    """Rows wide enough for the blocked sweep (n_r >= 2 x 512) with both phi directions
    active: each root's arithmetic must not depend on the thread slot the active list gives
    it, whose order follows shared-memory atomics."""
    f = synth.disc_field(700, 0.4, 0.1, 0.3, synth.stream_seed(14, k))
    m = 120
    outs = []
    for _ in range(3):
        fld = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, _opt(k))
        z, w, it = cc.critical_curves(fld, m, caustics=True, iters=True)
        outs.append((z, w, it))
    for z, w, it in outs[1:]:
        assert torch.equal(z, outs[0][0]) and torch.equal(w, outs[0][1]) and torch.equal(it, outs[0][2])
