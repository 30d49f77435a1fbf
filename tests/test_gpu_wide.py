"""Cluster tracing (several CTAs per phi sub-range, each updating a slice of the roots):
the chains match the FP64 oracle and the one-CTA tracer, for explicit cluster sizes on
small fields and for the automatic choice on a field with n_r >= 4096."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import cc, synth
from tests.gpu_util import compare_chain, match_row

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _solve(f, msteps, opt):
    field = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, opt)
    z, w, _ = cc.critical_curves(field, msteps, caustics=True)
    st, rep = cc.cc_field_report(field)
    return z.cpu().numpy(), w.cpu().numpy(), st, rep


@pytest.mark.parametrize("G", [2, 3, 8])
def test_cluster_tracer_matches_oracle(G):
    f = synth.disc_field(60, 0.4, 0.0, 0.4, synth.stream_seed(31, G), "loguniform", normalise=True)
    o = cc.cc_options_default()
    o.row_ctas = G
    zg, wg, st, rep = _solve(f, 200, o)
    assert st == cc.CC_OK and rep["uncertified"] == 0 and rep["seam_ambiguous"] == 0, rep
    zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 200)
    assert bad == 0
    worst, pairs = compare_chain(zg, zo, TOL)
    wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zg)
    assert np.abs(wg - wo).max() < TOL
    o1 = cc.cc_options_default()
    o1.row_ctas = 1
    z1, w1, st1, _ = _solve(f, 200, o1)
    compare_chain(zg, z1, 3e-10)


def test_cluster_tracer_rectangle():
    f = synth.rect_field(40, 0.4, 0.0, 0.35, synth.stream_seed(32, 0), 1.2, "loguniform")
    o = cc.rect_options(f.kappa_star, f.c1, f.c2)
    o.row_ctas = 4
    zg, wg, st, rep = _solve(f, 100, o)
    assert st == cc.CC_OK and rep["uncertified"] == 0, rep
    t = oracle.rect_choose_t(f.kappa_star, f.c1, f.c2)
    R = oracle.Rect(f.kappa_star, f.c1, f.c2, t)
    zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 100, rect=R)
    compare_chain(zg, zo, TOL)


def test_automatic_cluster_on_wide_rows():
    """n_r = 4200 >= 4096: clusters of 8 CTAs per sub-range by default."""
    n, msteps = 2100, 40
    f = synth.disc_field(n, 0.3, 0.1, 0.3, synth.stream_seed(33, 0), "loguniform", normalise=True)
    zg, wg, st, rep = _solve(f, msteps, cc.cc_options_default())
    assert st == cc.CC_OK and rep["uncertified"] == 0 and rep["seam_ambiguous"] == 0, rep
    for j in [0, msteps // 2, msteps]:
        zo, left = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, msteps))
        assert left == 0
        idx, dist, sep = match_row(zg[j], zo)
        assert dist < TOL and len(set(idx.tolist())) == len(idx)
        wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zg[j])
        assert np.abs(wg[j] - wo).max() < TOL


def test_automatic_single_cta_on_long_wide_chains():
    """n_r = 4200 >= 4096 with m >= 8 x the SM count: one CTA per sub-range (the root sum split
    then keeps warm rows cheap), its near positions in global memory (n_r above the shared
    tile); rows match the oracle."""
    n = 2100
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    msteps = 8 * sms + 2
    f = synth.disc_field(n, 0.3, 0.1, 0.3, synth.stream_seed(33, 1), "loguniform", normalise=True)
    zg, wg, st, rep = _solve(f, msteps, cc.cc_options_default())
    assert st == cc.CC_OK and rep["uncertified"] == 0 and rep["seam_ambiguous"] == 0, rep
    assert rep["subchains"] > 32  # one CTA per sub-range, not one cluster of 8
    assert rep["root_terms"] < 0.5 * rep["root_iterations"] * 2 * n
    for j in [0, msteps // 2 + 3, msteps]:
        zo, left = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, msteps))
        assert left == 0
        idx, dist, sep = match_row(zg[j], zo)
        assert dist < TOL and len(set(idx.tolist())) == len(idx)


def _fp64_opt(G):
    o = cc.cc_options_default()
    o.precision = cc.CC_FP64
    o.hp_arith = cc.CC_HP_FP64
    o.row_ctas = G
    return o


@pytest.mark.parametrize("G", [2, 8])
def test_fp64_cluster_tracer_matches_oracle(G):
    """The plain FP64 form traced by clusters of G CTAs per sub-range: chains and caustics
    match the oracle and the one-CTA FP64 form."""
    f = synth.disc_field(60, 0.4, 0.0, 0.4, synth.stream_seed(34, G), "loguniform", normalise=True)
    zg, wg, st, rep = _solve(f, 200, _fp64_opt(G))
    assert st == cc.CC_OK and rep["unconverged"] == 0 and rep["seam_ambiguous"] == 0, rep
    zo, _, bad = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 200)
    assert bad == 0
    compare_chain(zg, zo, TOL)
    wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zg)
    assert np.abs(wg - wo).max() < 1e-12 * (1 + np.abs(wo).max())
    z1, w1, st1, _ = _solve(f, 200, _fp64_opt(1))
    assert st1 == cc.CC_OK
    compare_chain(zg, z1, 2e-9)


def test_fp64_automatic_cluster_on_wide_rows():
    """The FP64 form on n_r = 4200 >= 4096 with few rows takes clusters of 8 CTAs by default;
    sampled rows pass the oracle's FP64 Newton check, points distinct."""
    from scipy.spatial import cKDTree
    n, msteps = 2100, 40
    f = synth.disc_field(n, 0.3, 0.1, 0.3, synth.stream_seed(33, 2), "loguniform", normalise=True)
    zg, wg, st, rep = _solve(f, msteps, _fp64_opt(0))
    assert st == cc.CC_OK and rep["unconverged"] == 0 and rep["seam_ambiguous"] == 0, rep
    step, wo = oracle.newton_check(f.x, f.y, f.m, f.kappa_s, f.gamma, msteps, zg)
    assert step.max() < TOL
    assert np.abs(wg - wo).max() < 1e-12 * (1 + np.abs(wo).max())
    for j in range(msteps + 1):
        pts = np.stack([zg[j].real, zg[j].imag], axis=1)
        d, nb = cKDTree(pts).query(pts, k=2)
        assert (d[:, 1] > 2 * TOL + step[j] + step[j][nb[:, 1]]).all(), j
