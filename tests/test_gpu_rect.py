"""Rectangular microlens field (Sec. 4.2, Appendices A and B) on the GPU against the FP64
oracle: n_r = 2N + t - 1 roots per row within 1e-9 theta_E, caustics of the GPU's points
within 1e-9 of the oracle's lens map, through the mixed, native-FP64-polish and plain FP64
forms, the far-field polish (N >= 128), the standalone caustic map and the batched launch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import cc, synth
from tests.gpu_util import compare_chain, match_row

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _field(n, kst, ks, g, aspect, seed):
    return synth.rect_field(n, kst, ks, g, synth.stream_seed(21, seed), aspect, "loguniform")


def _rect(f, t):
    return oracle.Rect(f.kappa_star, f.c1, f.c2, t)


def _solve(f, msteps, t=0, **kw):
    o = cc.rect_options(f.kappa_star, f.c1, f.c2, t)
    for k, v in kw.items():
        setattr(o, k, v)
    field = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, o)
    z, w, _ = cc.critical_curves(field, msteps, caustics=True)
    status, rep = cc.cc_field_report(field)
    return field, z.cpu().numpy(), w.cpu().numpy(), status, rep


@pytest.mark.parametrize("n,kst,ks,g,aspect,msteps", [
    (5, 0.3, 0.0, 0.2, 1.0, 200),
    (30, 0.4, 0.1, 0.35, 0.6, 100),
    (60, 0.5, 0.0, 0.5, 1.7, 64),
])
def test_rect_chain_matches_oracle(n, kst, ks, g, aspect, msteps):
    f = _field(n, kst, ks, g, aspect, n)
    t = oracle.rect_choose_t(kst, f.c1, f.c2)
    field, zg, wg, status, rep = _solve(f, msteps)
    assert field.n_roots == 2 * n + t - 1  # the library picks the same truncation order
    assert status == cc.CC_OK and rep["uncertified"] == 0, rep
    R = _rect(f, t)
    zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, ks, g, msteps, rect=R)
    assert bad == 0
    worst, pairs = compare_chain(zg, zo, TOL)
    # caustics: the oracle's lens map at the GPU's points (w is well conditioned in z on a
    # critical curve), and at the oracle's own points
    wo_at_g = oracle.map_caustics(f.x, f.y, f.m, ks, g, zg, rect=R)
    assert np.abs(wg - wo_at_g).max() < TOL
    wo = oracle.map_caustics(f.x, f.y, f.m, ks, g, zo, rect=R)
    for j, idx in enumerate(pairs):
        assert np.abs(wg[j] - wo[j][idx]).max() < 2 * TOL


def test_rect_far_field_polish_matches_oracle():
    """N >= 128: tracer far-field tables and local-expansion polish with the sheet polynomial."""
    n, kst, ks, g, msteps = 400, 0.45, 0.0, 0.4, 40
    f = _field(n, kst, ks, g, 1.3, 7)
    field, zg, wg, status, rep = _solve(f, msteps)
    assert status == cc.CC_OK and rep["uncertified"] == 0, rep
    t = oracle.rect_choose_t(kst, f.c1, f.c2)
    R = _rect(f, t)
    _, _, _, _, rep2 = _solve(f, msteps, far_field=0)
    for j in [0, msteps // 4, msteps // 2, msteps]:
        zo, left = oracle.solve_row(f.x, f.y, f.m, ks, g, oracle.phi(j, msteps), rect=R)
        assert left == 0
        idx, dist, sep = match_row(zg[j], zo)
        assert dist < TOL and len(set(idx.tolist())) == len(idx)
        wo = oracle.map_caustics(f.x, f.y, f.m, ks, g, zg[j], rect=R)
        assert np.abs(wg[j] - wo).max() < TOL


@pytest.mark.parametrize("kw", [dict(hp_arith=cc.CC_HP_FP64), dict(precision=cc.CC_FP64, hp_arith=cc.CC_HP_FP64)])
def test_rect_fp64_forms(kw):
    n, kst, ks, g, msteps = 12, 0.35, 0.05, 0.3, 64
    f = _field(n, kst, ks, g, 1.0, 3)
    field, zg, wg, status, rep = _solve(f, msteps, **kw)
    assert status == cc.CC_OK
    R = _rect(f, oracle.rect_choose_t(kst, f.c1, f.c2))
    zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, ks, g, msteps, rect=R)
    compare_chain(zg, zo, TOL)
    assert np.abs(wg - oracle.map_caustics(f.x, f.y, f.m, ks, g, zg, rect=R)).max() < TOL


def test_rect_standalone_caustic_map():
    n, kst, ks, g = 20, 0.4, 0.0, 0.3
    f = _field(n, kst, ks, g, 0.8, 11)
    t = 11
    o = cc.rect_options(kst, f.c1, f.c2, t)
    field = cc.cc_field_create(f.x, f.y, f.m, ks, g, o)
    rng = np.random.default_rng(0)
    z = (rng.uniform(-1.3, 1.3, 5000) * f.c1 + 1j * rng.uniform(-1.3, 1.3, 5000) * f.c2).astype(np.complex128)
    zt = torch.from_numpy(z).cuda()
    wt = torch.empty_like(zt)
    cc.cc_map_caustics(field, zt, wt)
    w = wt.cpu().numpy()
    wo = oracle.map_caustics(f.x, f.y, f.m, ks, g, z, rect=oracle.Rect(kst, f.c1, f.c2, t))
    assert np.abs(w - wo).max() < 1e-9 * (1 + np.abs(wo).max())


def test_rect_in_batch_equals_single():
    fields = [_field(40, 0.4, 0.0, 0.3, 1.0, 31), synth.disc_field(50, 0.4, 0.0, 0.3, synth.stream_seed(22, 1)),
              _field(150, 0.3, 0.1, 0.45, 1.5, 32)]
    handles, single = [], []
    for f in fields:
        o = cc.rect_options(f.kappa_star, f.c1, f.c2) if f.c1 > 0 else cc.cc_options_default()
        h = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, o)
        handles.append(h)
        z, w, _ = cc.critical_curves(h, 64, caustics=True)
        single.append((z.cpu().numpy(), w.cpu().numpy()))
    b = cc.batch_critical_curves(handles, [64] * len(fields), caustics=True)
    st, per, tot = cc.cc_batch_report(b)
    assert st == cc.CC_OK, tot
    for zb, wb, (zs, ws), h in zip(b.z, b.w, single, handles):
        zb, wb = zb.cpu().numpy(), wb.cpu().numpy()
        assert zb.shape == zs.shape == (65, h.n_roots)
        worst, pairs = compare_chain(zb, zs, 3e-10)
        for j, idx in enumerate(pairs):
            assert np.abs(wb[j] - ws[j][idx]).max() < 3e-10
