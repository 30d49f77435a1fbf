"""Parity at the full benchmark size, in the launch configuration bench.py times:
N = 1000 stars (log-uniform masses), m = 10^4 phi steps, 4096^2 maps over +-10.

The oracle cannot trace all 10^4 rows in test time, so it is compared on what it can
compute one by one:
- every one of the 2*10^7 critical points: the oracle's FP64 Newton correction |F/F'| at
  the GPU's point (the distance to the zero of F, to first order) and the oracle's lens
  map w at that point, against the GPU's caustic point; every row's points pairwise
  farther apart than their corrections (2N distinct zeros: the whole row's multiset);
- cold-solved sampled rows, matched root by root;
- whole pixel rows of the 4096^2 N_cc map, per-pixel winding numbers at sampled pixel
  centres, and the full distance map from the GPU's N_cc;
and Vieta's sums of the rationalised polynomial on every row."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import cc, synth
from tests.gpu_util import match_row

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def solved():
    wl = synth.workload_n1000()
    f = wl.fields[0]
    m = wl.msteps
    ext, px = wl.map_extent, wl.map_pixels
    field = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma)
    z, w, it = cc.critical_curves(field, m, caustics=True, iters=True)
    ncc = cc.crossing_map(w, -ext, ext, -ext, ext, px, px)
    d = cc.distance_map(ncc, 2 * ext / px)
    status, rep = cc.cc_field_report(field)
    return dict(f=f, m=m, ext=ext, px=px, z=z.cpu().numpy(), w=w.cpu().numpy(), it=it.cpu().numpy(),
                ncc=ncc.cpu().numpy(), d=d.cpu().numpy(), status=status, rep=rep)


def test_report_clean(solved):
    rep = solved["rep"]
    assert solved["status"] == cc.CC_OK, rep
    assert rep["unconverged"] == 0 and rep["uncertified"] == 0 and rep["seam_ambiguous"] == 0
    assert rep["max_err_est"] < 1e-10


def test_sampled_rows_match_cold_oracle(solved):
    f, m, z, w = solved["f"], solved["m"], solved["z"], solved["w"]
    u = synth.uniform(2024, 3)
    rows = sorted({0, 1, m // 2 - 1, m // 2, m // 2 + 1, m - 1, m} | {int(v * m) for v in u})
    for j in rows:
        zo, left = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, m))
        assert left == 0
        idx, dist, sep = match_row(z[j], zo)
        assert len(set(idx.tolist())) == len(idx), f"row {j}: pairing not 1:1"
        assert dist < TOL, f"row {j}: max |dz| = {dist}"
        assert dist < 1e-3 * sep
        wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zo[idx])
        assert np.abs(w[j] - wo).max() < TOL, f"row {j}: caustics"


def test_every_row_vieta_and_distinct(solved):
    """sum z = 2 sum z_i and sum z^2 = 2 sum z_i^2 - 2M/c_phi on all m+1 rows (a missing or
    doubled root moves these sums by O(1))."""
    f, m, z = solved["f"], solved["m"], solved["z"]
    zs = f.x + 1j * f.y
    phis = 2 * np.pi * np.arange(m + 1) / m
    c = f.gamma - (1 - f.kappa_s) * np.exp(-1j * phis)
    s1 = z.sum(axis=1)
    s2 = (z * z).sum(axis=1)
    assert np.abs(s1 - 2 * zs.sum()).max() < 1e-5
    assert np.abs(s2 - (2 * (zs * zs).sum() - 2 * f.m.sum() / c)).max() < 1e-4
    for j in range(0, m + 1, 997):
        row = np.sort_complex(z[j])
        assert oracle.min_separation(z[j]) > 1e-7


def test_every_point_newton_step_and_caustic(solved):
    """All (m+1) x 2N points at the library defaults (root_refresh = 64): the FP64 Newton
    correction is below 1e-9 everywhere, the caustic point is within 1e-9 of the oracle's
    lens map at the GPU's point, and within each row the points are pairwise farther apart
    than the sum of their corrections, so they are 2N distinct zeros (Sec. 3.2)."""
    from scipy.spatial import cKDTree
    f, m, z, w = solved["f"], solved["m"], solved["z"], solved["w"]
    step, wo = oracle.newton_check(f.x, f.y, f.m, f.kappa_s, f.gamma, m, z)
    worst = float(step.max())
    assert worst < TOL, f"largest Newton correction {worst:.3e} at {np.unravel_index(step.argmax(), step.shape)}"
    dw = float(np.abs(w - wo).max())
    assert dw < TOL, f"largest caustic difference {dw:.3e}"
    for j in range(m + 1):
        pts = np.stack([z[j].real, z[j].imag], axis=1)
        d, k = cKDTree(pts).query(pts, k=2)
        assert (d[:, 1] > 2 * TOL + step[j] + step[j][k[:, 1]]).all(), f"row {j}: two points share a zero"
    print(f"every point: max Newton correction {worst:.3e}, max caustic difference {dw:.3e}")


def test_whole_pixel_rows_match_oracle(solved):
    """16 whole rows of the 4096^2 N_cc map, bit for bit against the oracle's winding rule
    evaluated over all 2*10^7 GPU caustic segments (Sec. 5.1)."""
    w, ncc, ext, px = solved["w"], solved["ncc"], solved["ext"], solved["px"]
    u = synth.uniform(78, 16)
    rows = sorted({int((k + u[k]) * px / 16) for k in range(16)})
    ref = oracle.crossing_rows(w, -ext, ext, -ext, ext, px, px, rows)
    for t, r in enumerate(rows):
        bad = np.flatnonzero(ncc[r] != ref[t])
        assert bad.size == 0, f"row {r}: {bad.size} pixels differ, first at column {bad[:5]}"
    assert sum(int(np.abs(np.diff(ncc[r])).sum()) for r in rows) > 0  # the rows do cross caustics


def test_sampled_pixels_match_oracle_winding(solved):
    """N_cc at sampled pixel centres equals the oracle's per-point winding number over the
    same (GPU) caustic vertices, bit for bit."""
    w, ncc, ext, px = solved["w"], solved["ncc"], solved["ext"], solved["px"]
    u = synth.uniform(77, 2 * 48)
    for t in range(48):
        i, r = int(u[2 * t] * px), int(u[2 * t + 1] * px)
        pxc = oracle.pixel_center(-ext, ext, px, i)
        pyc = oracle.pixel_center(-ext, ext, px, r)
        assert ncc[r, i] == -oracle.winding_at(w, pxc, pyc), (r, i)
    assert ncc.min() >= 0


def test_full_distance_map_matches_oracle(solved):
    ncc, d, ext, px = solved["ncc"], solved["d"], solved["ext"], solved["px"]
    ref = oracle.distance_map(ncc, 2 * ext / px)
    assert np.array_equal(d, ref)
