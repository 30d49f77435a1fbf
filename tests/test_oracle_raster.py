"""Pins of the oracle's exact orientation predicate, Sunday winding numbers, N_cc maps and
distance maps: exact rational arithmetic, closed-form polygons, brute force, and the
physical identity that a caustic crossing creates or destroys a pair of images."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_02121_gb300 import synth
from tests import lensing_math as lm


def test_orient2d_matches_exact_rationals():
    u = synth.uniform(777, 6 * 4000)
    pts = (u.reshape(-1, 6) - 0.5) * 20
    for p in pts:
        assert oracle.orient2d(*p) == lm.orient_exact(*p)


def test_orient2d_near_degenerate():
    """Points on or within a few ulp of the line: the sign must still be exact."""
    rng = synth.uniform(778, 3 * 2000)
    cnt0 = 0
    for i in range(2000):
        ax, ay = 0.1 + rng[3 * i], -0.3
        bx, by = 3.7, 1.0 + rng[3 * i + 1]
        t = rng[3 * i + 2]
        cx = ax + t * (bx - ax)
        cy = ay + t * (by - ay)
        for k in (-2, -1, 0, 1, 2):
            cyk = cy + k * math.ulp(cy)
            s = oracle.orient2d(ax, ay, bx, by, cx, cyk)
            assert s == lm.orient_exact(ax, ay, bx, by, cx, cyk)
            cnt0 += s == 0
    # exactly collinear representable case
    assert oracle.orient2d(0.0, 0.0, 1.0, 1.0, 0.5, 0.5) == 0
    assert oracle.orient2d(0.0, 0.0, 1.0, 0.0, 0.5, 1e-300) == 1


def _circle(n, r, cx=0.0, cy=0.0, clockwise=True):
    t = np.arange(n + 1) * 2 * math.pi / n
    if clockwise:
        t = -t
    z = (cx + r * np.cos(t)) + 1j * (cy + r * np.sin(t))
    z[-1] = z[0]
    return z


def test_winding_clockwise_circle_counts_one_inside():
    """A clockwise polygon has winding number -1 inside (N_cc = +1), 0 outside; a
    counter-clockwise one +1 inside."""
    poly = _circle(64, 1.0)[:, None]  # one column = one closed chain
    ncc = oracle.crossing_map(poly, -2, 2, -2, 2, 40, 40)
    chord = 1.0 - math.cos(math.pi / 64)
    for r in range(40):
        for i in range(40):
            px = oracle.pixel_center(-2, 2, 40, i)
            py = oracle.pixel_center(-2, 2, 40, r)
            rho = math.hypot(px, py)
            if rho < 1.0 - chord - 1e-9:
                assert ncc[r, i] == 1
            elif rho > 1.0 + 1e-9:
                assert ncc[r, i] == 0
    ccw = _circle(64, 1.0, clockwise=False)[:, None]
    assert oracle.winding_at(ccw, 0.1, 0.2) == 1
    assert oracle.winding_at(poly, 0.1, 0.2) == -1


def test_crossing_map_equals_pointwise_winding():
    """The full-map routine makes the same decisions as the per-point definition."""
    u = synth.uniform(991, 2 * 31 * 3)
    w = ((u[0::2] - 0.5) * 5 + 1j * (u[1::2] - 0.5) * 5).reshape(31, 3)
    w[-1] = w[0]
    H, W = 23, 29
    ncc = oracle.crossing_map(w, -2.5, 2.5, -2.0, 2.7, W, H)
    for r in range(H):
        for i in range(W):
            px = oracle.pixel_center(-2.5, 2.5, W, i)
            py = oracle.pixel_center(-2.0, 2.7, H, r)
            assert ncc[r, i] == -oracle.winding_at(w, px, py)


def test_winding_half_open_rule_on_vertex_rows():
    """A vertex exactly on a pixel-centre row is counted once (half-open y rule)."""
    # square with vertices on the line y = 0 (a pixel-centre row below)
    sq = np.array([-1 - 1j, -1 + 1j, 1 + 1j, 1 - 1j, -1 - 1j])[:, None]  # clockwise
    for py in (-1.0, 0.0, 0.5, 1.0):
        wn = oracle.winding_at(sq, 0.0, py)
        assert wn == (-1 if -1.0 <= py < 1.0 else 0)


@pytest.mark.parametrize("kappa_s,gamma", [(0.0, 0.3), (0.25, 0.4)])
def test_chang_refsdal_ncc_is_one_inside(kappa_s, gamma):
    """N_cc = 1 inside the Chang-Refsdal caustic and 0 outside, away from the curve."""
    x, y, m = np.array([0.0]), np.array([0.0]), np.array([1.0])
    z, _, _ = oracle.critical_curves(x, y, m, kappa_s, gamma, 2000)
    w = oracle.map_caustics(x, y, m, kappa_s, gamma, z)
    ext = 1.2
    H = W = 48
    ncc = oracle.crossing_map(w, -ext, ext, -ext, ext, W, H)
    assert ncc.min() >= 0 and ncc.max() >= 1
    # compare with image counts at pixel centres well away from the caustic
    caus = w[:-1].ravel()
    rng = synth.uniform(4242, 2 * 60)
    checked = 0
    for t in range(60):
        i = int(rng[2 * t] * W)
        r = int(rng[2 * t + 1] * H)
        px = oracle.pixel_center(-ext, ext, W, i)
        py = oracle.pixel_center(-ext, ext, H, r)
        if np.min(np.abs(caus - complex(px, py))) < 0.02:
            continue
        nimg = lm.image_count(x, y, m, kappa_s, gamma, complex(px, py))
        assert nimg == 2 + 2 * ncc[r, i], (px, py, nimg, ncc[r, i])
        checked += 1
    assert checked > 20


@pytest.mark.parametrize("sep", [0.6, 1.8, 4.0])
def test_binary_ncc_matches_image_counts(sep):
    """Two unit masses: the number of images of a point source is 3 + 2 N_cc."""
    x = np.array([-sep / 2, sep / 2])
    y = np.array([0.05, -0.05])
    m = np.ones(2)
    kappa_s, gamma = 0.0, 0.1
    z, _, bad = oracle.critical_curves(x, y, m, kappa_s, gamma, 1000)
    assert bad == 0
    w = oracle.map_caustics(x, y, m, kappa_s, gamma, z)
    ext = 2.5
    H = W = 40
    ncc = oracle.crossing_map(w, -ext, ext, -ext, ext, W, H)
    assert ncc.min() >= 0
    caus = w[:-1].ravel()
    checked = 0
    for r in range(0, H, 3):
        for i in range(0, W, 3):
            px = oracle.pixel_center(-ext, ext, W, i)
            py = oracle.pixel_center(-ext, ext, H, r)
            if np.min(np.abs(caus - complex(px, py))) < 0.03:
                continue
            nimg = lm.image_count(x, y, m, kappa_s, gamma, complex(px, py))
            assert nimg == 3 + 2 * ncc[r, i], (px, py, nimg, ncc[r, i])
            checked += 1
    assert checked > 50


def test_distance_single_feature_closed_form():
    ncc = np.zeros((9, 11), dtype=np.int32)
    ncc[4, 6] = 1  # the pixel and its 4 neighbours are features
    d = oracle.distance_map(ncc, 0.5, method="separable")
    db = oracle.distance_map(ncc, 0.5, method="brute")
    feats = [(4, 6), (3, 6), (5, 6), (4, 5), (4, 7)]
    for r in range(9):
        for i in range(11):
            ref = 0.5 * min(math.sqrt((r - fr) ** 2 + (i - fi) ** 2) for fr, fi in feats)
            assert d[r, i] == ref
            assert db[r, i] == ref


def test_distance_no_feature_is_infinite():
    d = oracle.distance_map(np.full((5, 7), 3, dtype=np.int32), 1.0)
    assert np.all(np.isinf(d))


@pytest.mark.parametrize("seed,H,W", [(1, 17, 23), (2, 40, 33), (3, 64, 64), (4, 1, 50), (5, 50, 1)])
def test_distance_separable_equals_brute(seed, H, W):
    u = synth.uniform(5000 + seed, H * W).reshape(H, W)
    ncc = (u > 0.97).astype(np.int32)
    ncc[: H // 3, : W // 2] += 1
    a = oracle.distance_map(ncc, 0.01, method="separable")
    b = oracle.distance_map(ncc, 0.01, method="brute")
    assert np.array_equal(a, b)
    mask = oracle.feature_mask(ncc)
    assert np.all((a == 0) == (mask == 1))


def test_point_on_edge_not_counted():
    """A pixel centre exactly on an edge (orientation 0) is neither left nor right of it:
    on the clockwise square's upward left edge only the downward right edge counts, on the
    downward right edge nothing counts."""
    sq = np.array([-1 - 1j, -1 + 1j, 1 + 1j, 1 - 1j, -1 - 1j])[:, None]
    assert oracle.winding_at(sq, -1.0, 0.25) == -1
    assert oracle.winding_at(sq, 1.0, 0.25) == 0
    assert oracle.winding_at(sq, -1.0 - 1e-12, 0.25) == 0
    assert oracle.winding_at(sq, 1.0 - 1e-12, 0.25) == -1


@pytest.mark.parametrize("angle", [0.0, math.pi / 2, math.pi, 3 * math.pi / 2])
def test_moving_distance_axis_aligned_equals_row_scan(angle):
    """Along the axes the traversal visits the pixels of one row or column in order: the
    distance is pixel * (k - 0.5) for the k-th pixel ahead, k = 1, 2, ..."""
    u = synth.uniform(600 + int(angle * 10), 23 * 31).reshape(23, 31)
    ncc = (u > 0.93).astype(np.int32)
    feat = oracle.feature_mask(ncc).astype(bool)
    d = oracle.moving_distance_map(ncc, 0.5, angle)
    H, W = ncc.shape
    dx, dy = round(math.cos(angle)), round(math.sin(angle))
    for r in range(H):
        for i in range(W):
            if feat[r, i]:
                assert d[r, i] == 0.0
                continue
            k, x, y, ref = 0, i, r, math.inf
            while True:
                x, y, k = x + dx, y + dy, k + 1
                if not (0 <= x < W and 0 <= y < H):
                    break
                if feat[y, x]:
                    ref = 0.5 * (k - 0.5)
                    break
            assert d[r, i] == pytest.approx(ref, rel=1e-6) or (math.isinf(ref) and math.isinf(d[r, i]))


@pytest.mark.parametrize("angle", [0.3, 1.1, 2.0, 4.0, 5.5])
def test_moving_distance_to_a_feature_line_closed_form(angle):
    """A caustic along one full pixel column i0 (features at columns i0-1..i0+1 after the
    4-neighbour rule): a ray from (i + 0.5, r + 0.5) with cos > 0 first enters column i0 - 1
    at t = (i0 - 1 - i - 0.5) / cos, in pixel units, if it is still inside the map there."""
    H, W, i0 = 40, 50, 30
    ncc = np.zeros((H, W), dtype=np.int32)
    ncc[:, i0:] = 1  # boundary between columns i0-1 and i0: features i0-1 and i0
    d = oracle.moving_distance_map(ncc, 1.0, angle)
    c, s = math.cos(angle), math.sin(angle)
    for r in range(H):
        for i in range(i0 - 1):
            if c <= 0:
                assert math.isinf(d[r, i])
                continue
            t = (i0 - 1 - i - 0.5) / c
            yend = r + 0.5 + t * s
            if 0.0 < yend < H - 1e-6 and abs(yend - round(yend)) > 1e-4:
                assert d[r, i] == pytest.approx(t, rel=1e-5, abs=1e-5)


def test_crossing_rows_equal_pointwise_winding():
    """Listed rows make the per-point decisions at the full grid's own pixel centres."""
    u = synth.uniform(992, 2 * 41 * 4)
    w = ((u[0::2] - 0.5) * 5 + 1j * (u[1::2] - 0.5) * 5).reshape(41, 4)
    w[-1] = w[0]
    H, W = 37, 19
    for rows in [[0, 1, 2, 3, 4], [11], [36, 30, 7], []]:
        out = oracle.crossing_rows(w, -2.5, 2.5, -2.2, 2.6, W, H, rows)
        assert out.shape == (len(rows), W)
        for t, r in enumerate(rows):
            py = oracle.pixel_center(-2.2, 2.6, H, r)
            for i in range(W):
                px = oracle.pixel_center(-2.5, 2.5, W, i)
                assert out[t, i] == -oracle.winding_at(w, px, py)
    with pytest.raises(ValueError):
        oracle.crossing_rows(w, -2.5, 2.5, -2.2, 2.6, W, H, [5, 37])
