"""GPU-vs-oracle parity through the C ABI: critical points and caustics within 1e-9
theta_E of the FP64 oracle, crossing counts and distance maps bit-exact."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2506_02121_gb300 import cc, synth
from tests import lensing_math as lm
from tests.gpu_util import compare_chain, match_row

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _opts(**kw):
    o = cc.cc_options_default()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _solve(x, y, m_, ks, g, msteps, **kw):
    field = cc.cc_field_create(x, y, m_, ks, g, _opts(**kw))
    z, w, it = cc.critical_curves(field, msteps, caustics=True, iters=True)
    status, rep = cc.cc_field_report(field)
    return z.cpu().numpy(), w.cpu().numpy(), it.cpu().numpy(), status, rep


def _check_against_oracle(x, y, m_, ks, g, msteps, **kw):
    zg, wg, it, status, rep = _solve(x, y, m_, ks, g, msteps, **kw)
    assert status == cc.CC_OK, str(rep)
    zo, _, bad = oracle.critical_curves(x, y, m_, ks, g, msteps)
    assert bad == 0
    worst, pairs = compare_chain(zg, zo, TOL)
    wo = oracle.map_caustics(x, y, m_, ks, g, zo)
    wworst = 0.0
    for j, idx in enumerate(pairs):
        wworst = max(wworst, float(np.abs(wg[j] - wo[j][idx]).max()))
    assert wworst < TOL, f"caustics differ by {wworst}"
    assert it.min() >= 0
    return worst, wworst, rep


def test_small_field_mixed():
    f = synth.workload_small().fields[0]
    worst, wworst, rep = _check_against_oracle(f.x, f.y, f.m, f.kappa_s, f.gamma, 1000)
    assert rep["unconverged"] == 0 and rep["uncertified"] == 0 and rep["seam_ambiguous"] == 0


def test_small_field_fp64():
    f = synth.workload_small().fields[0]
    _check_against_oracle(f.x, f.y, f.m, f.kappa_s, f.gamma, 1000, precision=cc.CC_FP64, hp_arith=cc.CC_HP_FP64)


def test_small_field_mixed_native_fp64_polish():
    f = synth.workload_small().fields[0]
    _check_against_oracle(f.x, f.y, f.m, f.kappa_s, f.gamma, 200, hp_arith=cc.CC_HP_FP64)


@pytest.mark.parametrize("n,msteps,subchains,ks,g,mass", [
    (1, 2, 0, 0.0, 0.3, "unit"),
    (1, 64, 3, 0.3, 1.3, "unit"),
    (2, 10, 1, 0.0, 0.1, "loguniform"),
    (3, 98, 7, 0.2, 0.6, "loguniform"),
    (17, 40, 0, 0.1, 0.05, "unit"),
    (33, 26, 13, 0.0, 0.45, "loguniform"),
])
def test_ragged_sizes(n, msteps, subchains, ks, g, mass):
    f = synth.disc_field(n, 0.3, ks, g, synth.stream_seed(9, n), mass)
    _check_against_oracle(f.x, f.y, f.m, ks, g, msteps, subchains=subchains)


def test_no_predictor_and_small_blocks():
    f = synth.disc_field(40, 0.5, 0.1, 0.3, synth.stream_seed(10, 1), "loguniform")
    _check_against_oracle(f.x, f.y, f.m, 0.1, 0.3, 60, predictor=0, block_threads=64)


@pytest.mark.parametrize("sep,loops", [(0.6, 3), (1.8, 1), (4.0, 2)])
def test_binary_topology_from_gpu_chains(sep, loops):
    """Chains joined across sub-ranges still close into 3 / 1 / 2 loops."""
    x = np.array([-sep / 2, sep / 2])
    zg, _, _, status, rep = _solve(x, np.zeros(2), np.ones(2), 0.0, 0.0, 400, subchains=8)
    assert status == cc.CC_OK and rep["seam_ambiguous"] == 0
    found, _ = lm.join_chains(zg)
    assert len(found) == loops
    # each chain is continuous: consecutive rows move by much less than the root spacing
    steps = np.abs(np.diff(zg, axis=0))
    assert steps.max() < 0.2


def test_chains_continuous_across_seams():
    f = synth.disc_field(60, 0.4, 0.0, 0.4, synth.stream_seed(11, 0), "loguniform")
    zg, _, _, status, rep = _solve(f.x, f.y, f.m, 0.0, 0.4, 2000, subchains=16)
    assert status == cc.CC_OK and rep["seam_ambiguous"] == 0
    zo, _, _ = oracle.critical_curves(f.x, f.y, f.m, 0.0, 0.4, 2000)
    # same chain decomposition: per-step jumps of the GPU chains are as small as the oracle's
    assert np.abs(np.diff(zg, axis=0)).max() <= 1.01 * np.abs(np.diff(zo, axis=0)).max() + 1e-12


def test_map_caustics_standalone():
    f = synth.workload_small().fields[0]
    u = synth.uniform(123, 2 * 5000)
    z = (u[0::2] - 0.5) * 12 + 1j * (u[1::2] - 0.5) * 12
    zs = f.x + 1j * f.y
    z = z[np.min(np.abs(z[:, None] - zs[None, :]), axis=1) > 0.05]
    for hp in (cc.CC_HP_DFLOAT, cc.CC_HP_FP64):
        field = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma, _opts(hp_arith=hp))
        zt = torch.from_numpy(z).cuda()
        wt = torch.empty_like(zt)
        cc.cc_map_caustics(field, zt, wt)
        wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, z)
        assert np.abs(wt.cpu().numpy() - wo).max() < TOL


def test_crossing_map_bit_exact_on_oracle_vertices():
    f = synth.workload_small().fields[0]
    zo, _, _ = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 1000)
    wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zo)
    ref = oracle.crossing_map(wo, -3, 3, -3, 3, 256, 256)
    got = cc.crossing_map(torch.from_numpy(wo).cuda(), -3, 3, -3, 3, 256, 256).cpu().numpy()
    assert np.array_equal(got, ref)
    assert ref.max() >= 1 and ref.min() >= 0


@pytest.mark.parametrize("W,H", [(1, 1), (1, 37), (29, 1), (33, 17), (64, 65)])
def test_crossing_map_ragged_grids(W, H):
    u = synth.uniform(400 + W + H, 2 * 41 * 5)
    w = ((u[0::2] - 0.5) * 6 + 1j * (u[1::2] - 0.5) * 6).reshape(41, 5)
    ref = oracle.crossing_map(w, -2.0, 2.5, -2.2, 1.9, W, H)
    got = cc.crossing_map(torch.from_numpy(w).cuda(), -2.0, 2.5, -2.2, 1.9, W, H).cpu().numpy()
    assert np.array_equal(got, ref)


def test_crossing_map_vertices_on_pixel_centres():
    """Vertices and edges through pixel centres exercise the exact predicate and the
    half-open row rule."""
    W = H = 16
    xs = [oracle.pixel_center(-1, 1, W, i) for i in range(W)]
    ys = [oracle.pixel_center(-1, 1, H, r) for r in range(H)]
    poly = np.array([xs[2] + 1j * ys[3], xs[2] + 1j * ys[12], xs[13] + 1j * ys[12], xs[13] + 1j * ys[3],
                     xs[7] + 1j * ys[7], xs[2] + 1j * ys[3]])
    w = np.stack([poly, poly[::-1]], axis=1)  # clockwise and counter-clockwise copies
    w2 = poly[:, None]
    for ww in (w, w2):
        ref = oracle.crossing_map(ww, -1, 1, -1, 1, W, H)
        got = cc.crossing_map(torch.from_numpy(np.ascontiguousarray(ww)).cuda(), -1, 1, -1, 1, W, H).cpu().numpy()
        assert np.array_equal(got, ref)


def test_crossing_map_long_and_outside_segments():
    w = np.array([[-50 - 50j, 0.1 + 0j], [50 + 40j, 30 + 0.5j], [-50 + 60j, 0.2 + 1j], [-50 - 50j, 0.1 + 0j]])
    ref = oracle.crossing_map(w, -1, 1, -1, 1, 40, 30)
    got = cc.crossing_map(torch.from_numpy(w).cuda(), -1, 1, -1, 1, 40, 30).cpu().numpy()
    assert np.array_equal(got, ref)
    empty = torch.zeros((1, 3), dtype=torch.complex128, device="cuda")
    assert int(cc.crossing_map(empty, -1, 1, -1, 1, 8, 8).abs().sum()) == 0


def test_crossing_map_near_ties_tiny_and_huge_segments():
    """Segments whose crossings fall within 1e-12 to 1e-3 pixel of pixel centres, segments far
    shorter than FP32 can resolve at |w| ~ 10, vertices with +0 and -0 ordinates, and
    coordinates beyond 2^100 (up to 1e140): the FP32 fast path must hand every undecidable
    pair to the exact predicate, and the counts stay equal to the oracle's."""
    W = H = 512
    x0, x1, y0, y1 = -10.0, 10.0, -10.0, 10.0
    u = synth.uniform(4711, 6 * 3000)
    cols = []
    for t in range(3000):
        r = int(u[6 * t] * H)
        i = int(u[6 * t + 1] * W)
        px = oracle.pixel_center(x0, x1, W, i)
        py = oracle.pixel_center(y0, y1, H, r)
        off = (u[6 * t + 2] - 0.5) * 10 ** (-12 + 9 * u[6 * t + 3]) * (x1 - x0) / W
        length = 10 ** (-9 + 7 * u[6 * t + 4])
        ang = 0.05 + 3.0 * u[6 * t + 5]
        d = length * np.exp(1j * ang)
        c = complex(px + off, py)
        cols.append([c - 0.37 * d, c + 0.63 * d, c + 0.63 * d + 0.5 * length, c - 0.37 * d])
    w = np.array(cols).T.copy()
    ref = oracle.crossing_map(w, x0, x1, y0, y1, W, H)
    got = cc.crossing_map(torch.from_numpy(w).cuda(), x0, x1, y0, y1, W, H).cpu().numpy()
    assert np.array_equal(got, ref)
    # +0 / -0 ordinates, a vertical edge through pixel centres, and huge coordinates
    z0 = np.array([complex(0.0, 0.0), complex(0.3, -0.0), complex(0.3, 0.7), complex(0.0, 0.0)])
    # (products of coordinate differences must stay inside the double range, |w| < 1e154, for
    # the exact orientation predicate on either side)
    big = np.array([complex(-3e30, -0.25), complex(4e30, 0.75), complex(1e140, -1e140), complex(-3e30, -0.25)])
    for ww in (z0[:, None], big[:, None], np.stack([z0, big], axis=1)):
        ww = np.ascontiguousarray(ww)
        ref = oracle.crossing_map(ww, -1, 1, -1, 1, 64, 48)
        got = cc.crossing_map(torch.from_numpy(ww).cuda(), -1, 1, -1, 1, 64, 48).cpu().numpy()
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("W,H,density", [(1, 1, 0.0), (1, 50, 0.05), (50, 1, 0.05), (64, 48, 0.01),
                                         (200, 130, 0.001), (97, 101, 0.0),
                                         # several 64-row feature words per column, ragged last word
                                         (333, 321, 0.0005), (64, 64, 0.3), (31, 257, 0.002),
                                         # distances beyond the square-root table (d^2 >= 2^16)
                                         (700, 650, 0.000004),
                                         # 16-bit hull stacks (W > 8192), and the wide-map path (W > 32768)
                                         (9000, 5, 0.001), (33000, 3, 0.0005)])
def test_distance_map_bit_exact(W, H, density):
    u = synth.uniform(77 + W * H, W * H).reshape(H, W)
    ncc = (u < density).astype(np.int32)
    ncc[: H // 2, : W // 3] += 2 if density > 0 else 0
    ref = oracle.distance_map(ncc, 0.0123)
    got = cc.distance_map(torch.from_numpy(ncc).cuda(), 0.0123).cpu().numpy()
    assert np.array_equal(got, ref)


def test_distance_map_single_feature_and_checkerboard():
    """A lone feature (distances up to the far corner, every column's nearest feature in
    another 64-row word) and a map where every pixel is a feature."""
    H, W = 517, 389
    ncc = np.zeros((H, W), dtype=np.int32)
    ncc[200, 100] = 1
    ref = oracle.distance_map(ncc, 0.5)
    got = cc.distance_map(torch.from_numpy(ncc).cuda(), 0.5).cpu().numpy()
    assert np.array_equal(got, ref)
    cb = (np.add.outer(np.arange(70), np.arange(90)) % 2).astype(np.int32)
    got = cc.distance_map(torch.from_numpy(cb).cuda(), 0.25).cpu().numpy()
    assert np.array_equal(got, oracle.distance_map(cb, 0.25)) and got.max() == 0.0


def test_degenerate_and_invalid_arguments():
    f = synth.workload_small().fields[0]
    field = cc.cc_field_create(f.x, f.y, f.m, f.kappa_s, f.gamma)
    z = torch.empty((12, field.n_roots), dtype=torch.complex128, device="cuda")
    with pytest.raises(cc.CCError) as e:
        cc.cc_critical_curves(field, 11, z, workspace=cc.workspace(16))
    assert e.value.status == cc.CC_EINVAL
    z = torch.empty((11, field.n_roots), dtype=torch.complex128, device="cuda")
    with pytest.raises(cc.CCError) as e:
        cc.cc_critical_curves(field, 10, z, workspace=cc.workspace(16))
    assert e.value.status == cc.CC_ENOMEM
    with pytest.raises(cc.CCError):
        cc.crossing_map(torch.zeros((2, 2), dtype=torch.complex128, device="cuda"), 1, -1, 0, 1, 4, 4)


def test_device_star_arrays_accepted():
    f = synth.workload_small().fields[0]
    field = cc.cc_field_create(torch.from_numpy(f.x).cuda(), torch.from_numpy(f.y).cuda(),
                               torch.from_numpy(f.m).cuda(), f.kappa_s, f.gamma)
    z, _, _ = cc.critical_curves(field, 20, caustics=False)
    zo, _, _ = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 20)
    compare_chain(z.cpu().numpy(), zo, TOL)


@pytest.mark.parametrize("angle", [0.0, 0.7, math.pi / 2, 2.5, math.pi, 4.4, 3 * math.pi / 2, 6.0])
def test_moving_distance_map_bit_exact(angle):
    u = synth.uniform(900 + int(10 * angle), 70 * 90).reshape(70, 90)
    ncc = (u < 0.004).astype(np.int32)
    ncc[20:45, 10:60] += 1
    ref = oracle.moving_distance_map(ncc, 0.02, angle)
    got = cc.moving_distance_map(torch.from_numpy(ncc).cuda(), 0.02, angle).cpu().numpy()
    assert np.array_equal(got, ref)


def test_moving_distance_map_on_real_caustics():
    f = synth.workload_small().fields[0]
    zo, _, _ = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 400)
    wo = oracle.map_caustics(f.x, f.y, f.m, f.kappa_s, f.gamma, zo)
    ncc = oracle.crossing_map(wo, -3, 3, -3, 3, 128, 128)
    for angle in (0.25, 1.9):
        ref = oracle.moving_distance_map(ncc, 6 / 128, angle)
        got = cc.moving_distance_map(torch.from_numpy(ncc).cuda(), 6 / 128, angle).cpu().numpy()
        assert np.array_equal(got, ref)
        assert np.isfinite(ref).any() and np.isinf(ref).any()


@pytest.mark.parametrize("n,msteps,ks,g", [(400, 300, 0.0, 0.35), (1500, 40, 0.2, 0.55)])
def test_far_field_polish_matches_oracle_and_direct(n, msteps, ks, g):
    """The local-expansion polish (stars beyond a 5x5 block of cells through 32-term local
    expansions) agrees with the oracle and with the all-direct polish within 1e-9."""
    f = synth.disc_field(n, 0.45, ks, g, synth.stream_seed(12, n), "loguniform", normalise=True)
    zf, wf, _, st, rep = _solve(f.x, f.y, f.m, ks, g, msteps)
    assert st == cc.CC_OK and rep["uncertified"] == 0, rep
    zd, wd, _, st2, rep2 = _solve(f.x, f.y, f.m, ks, g, msteps, far_field=0)
    assert st2 == cc.CC_OK
    # each side is certified to 1e-10 (tol_cert), so the root sets agree to twice that plus
    # rounding (the column labelling may differ: chains follow the tracer's own trajectory)
    worst, pairs = compare_chain(zf, zd, 3e-10)
    for j, idx in enumerate(pairs):
        assert np.abs(wf[j] - wd[j][idx]).max() < 3e-10
    rows = [0, msteps // 3, msteps // 2, msteps]
    for j in rows:
        zo, left = oracle.solve_row(f.x, f.y, f.m, ks, g, oracle.phi(j, msteps))
        idx, dist, sep = match_row(zf[j], zo)
        assert dist < TOL and len(set(idx.tolist())) == len(idx)
        wo = oracle.map_caustics(f.x, f.y, f.m, ks, g, zo[idx])
        assert np.abs(wf[j] - wo).max() < TOL
