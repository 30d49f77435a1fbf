"""Parity at the largest single-field size: N = 20000 stars (Kroupa-like masses in
[0.08, 1.5], kappa_* = 0.2, kappa_s = 0.3, gamma = 0.3), m = 2*10^4 phi steps
(8.0*10^8 root points), an 8192^2 crossing map and its distance map over +-10, through the
same single-field calls as the benchmark step.

The oracle cannot solve rows of 40000 roots cold in test time, so it checks what it can
compute one by one:
- at sampled roots of sampled rows, the FP64 Newton step |F/F'| (to first order the
  distance to the zero, for a simple root) and the lens map w;
- one whole row refined by the oracle's own Aberth iteration started from the GPU's roots
  (its repulsion term would push a doubled root towards the zero it missed);
- the winding number at sampled pixel centres over all 8*10^8 GPU caustic segments;
- the full distance map from the GPU's N_cc.
Vieta's sums of the rationalised polynomial are checked on every row: a missing or doubled
root moves the first one by the distance between two zeros."""
import concurrent.futures
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import cc, synth

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def solved():
    wl = synth.workload_n20000()
    f = wl.fields[0]
    m, ext, px = wl.msteps, wl.map_extent, wl.map_pixels
    field = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma)
    z, w, _ = cc.critical_curves(field, m, caustics=True)
    ncc = cc.crossing_map(w, -ext, ext, -ext, ext, px, px)
    d = cc.distance_map(ncc, 2 * ext / px)
    torch.cuda.synchronize()
    status, rep = cc.cc_field_report(field)
    yield dict(f=f, m=m, ext=ext, px=px, z=z, w=w, ncc=ncc.cpu().numpy(), d=d.cpu().numpy(), status=status,
               rep=rep)
    del z, w, ncc, d, field
    torch.cuda.empty_cache()


def test_report_clean(solved):
    rep = solved["rep"]
    assert solved["status"] == cc.CC_OK, rep
    assert rep["unconverged"] == 0 and rep["uncertified"] == 0 and rep["seam_ambiguous"] == 0
    assert rep["max_err_est"] < 1e-10
    assert solved["z"].shape == (solved["m"] + 1, 40000)


def test_every_row_vieta(solved):
    """sum z = 2 sum z_i and sum z^2 = 2 sum z_i^2 - 2M/c_phi, c_phi = gamma - (1 - kappa_s)
    e^{-i phi}, on all 20001 rows (sums taken on the device in FP64)."""
    f, m, z = solved["f"], solved["m"], solved["z"]
    nr = z.shape[1]
    zs = f.x + 1j * f.y
    phis = np.array([oracle.phi(j, m) for j in range(m + 1)])
    c = f.gamma - (1 - f.kappa_s) * np.exp(-1j * phis)
    s1 = z.sum(dim=1).cpu().numpy()
    s2 = (z * z).sum(dim=1).cpu().numpy()
    a1 = z.abs().sum(dim=1).cpu().numpy()
    zmax = float(z.abs().max())
    # each root is within 1e-10 (certified); FP64 rounding of the sums on top
    tol1 = 2e-10 * nr + 1e-13 * a1
    tol2 = 4e-10 * nr * zmax + 1e-13 * a1 * zmax
    assert np.all(np.abs(s1 - 2 * zs.sum()) < tol1)
    assert np.all(np.abs(s2 - (2 * (zs * zs).sum() - 2 * f.m.sum() / c)) < tol2)


def _rows(m):
    u = synth.uniform(4242, 5)
    return sorted({0, 1, m // 2, m - 1, m} | {int(v * m) for v in u})


def test_sampled_roots_are_fp64_zeros_and_map_to_oracle_caustics(solved):
    f, m, z, w = solved["f"], solved["m"], solved["z"], solved["w"]
    nr = z.shape[1]
    for j in _rows(m):
        zr = z[j].cpu().numpy()
        wr = w[j].cpu().numpy()
        ks = np.unique((synth.uniform(9000 + j, 400) * nr).astype(np.int64))
        ph = oracle.phi(j, m)
        for k in ks:
            step = oracle.F(f.x, f.y, f.m, f.kappa_s, f.gamma, ph, zr[k]) / oracle.dF(f.x, f.y, f.m, zr[k])
            assert abs(step) < TOL, (j, int(k), abs(step))
        wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zr[ks])
        assert np.abs(wr[ks] - wo).max() < TOL, j


def test_one_row_refined_by_oracle_aberth_and_distinct(solved):
    f, m, z = solved["f"], solved["m"], solved["z"]
    j = m // 4 + 7
    zr = z[j].cpu().numpy()
    zo, left = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, m), z0=zr)
    assert left == 0
    assert np.abs(zo - zr).max() < TOL
    assert oracle.min_separation(zr) > 1e-7


def test_sampled_pixels_match_oracle_winding(solved):
    """N_cc at sampled pixel centres equals minus the oracle's winding number over every
    segment of the GPU's caustics, bit for bit.  The segments are visited in chunks of rows
    (consecutive chunks share their boundary row), each pixel's sum in its own thread."""
    w, ncc, ext, px, m = solved["w"], solved["ncc"], solved["ext"], solved["px"], solved["m"]
    u = synth.uniform(78, 2 * 6)
    pix = [(int(u[2 * t] * px), int(u[2 * t + 1] * px)) for t in range(6)]
    hot = np.argwhere(ncc == ncc.max())[0]
    pix += [(int(hot[1]), int(hot[0])), (px // 2, px // 2)]
    centres = [(oracle.pixel_center(-ext, ext, px, i), oracle.pixel_center(-ext, ext, px, r)) for i, r in pix]
    wn = [0] * len(pix)
    chunk = 1000
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(pix), os.cpu_count() or 1)) as ex:
        for j0 in range(0, m, chunk):
            wc = w[j0:min(j0 + chunk, m) + 1].cpu().numpy()
            for t, s in enumerate(ex.map(lambda c: oracle.winding_at(wc, c[0], c[1]), centres)):
                wn[t] += s
    for (i, r), v in zip(pix, wn):
        assert ncc[r, i] == -v, (r, i)
    assert ncc.max() > 0 and ncc.min() >= 0


def test_full_distance_map_matches_oracle(solved):
    ncc, d, ext, px = solved["ncc"], solved["d"], solved["ext"], solved["px"]
    ref = oracle.distance_map(ncc, 2 * ext / px)
    assert np.array_equal(d, ref)
