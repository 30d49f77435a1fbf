"""Pins of the FP64 oracle's critical points and caustics against mathematics it does not
share: closed forms, polynomial identities, brute-force companion roots, finite-difference
Jacobians and the known two-point-mass topologies."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_02121_gb300 import synth
from tests import lensing_math as lm


def _random_field(n, seed, spread=3.0, mass="unit"):
    u = synth.uniform(seed, 3 * n)
    x = spread * (2 * u[0::3] - 1)
    y = spread * (2 * u[1::3] - 1)
    m = np.ones(n) if mass == "unit" else 0.2 + 1.3 * u[2::3]
    return x, y, m


@pytest.mark.parametrize("kappa_s", [0.0, 0.3])
@pytest.mark.parametrize("gamma", [0.2, 0.5, 1.3])
def test_chang_refsdal_closed_form(kappa_s, gamma):
    """One star with shear: every row matches z0 +- sqrt(m / ((1-kappa_s)e^{-i phi} - gamma))."""
    x, y, m = np.array([0.7]), np.array([-0.4]), np.array([0.6])
    for msteps in (2, 64):  # m = 2: phase steps of pi, the warm start of Sec. 3.2 stalls
        z, it, bad = oracle.critical_curves(x, y, m, kappa_s, gamma, msteps)
        assert bad == 0
        for j in range(msteps + 1):
            ref = lm.chang_refsdal_roots(complex(x[0], y[0]), m[0], kappa_s, gamma, oracle.phi(j, msteps))
            err, _ = lm.match_rows(z[j], ref)
            assert err < 1e-12


@pytest.mark.parametrize("kappa_s,gamma", [(0.0, 0.2), (0.3, 0.5), (0.0, 1.3)])
def test_chang_refsdal_caustic_closed_form(kappa_s, gamma):
    x, y, m = np.array([0.7]), np.array([-0.4]), np.array([0.6])
    for j in [0, 5, 17, 32]:
        ph = oracle.phi(j, 64)
        zc = lm.chang_refsdal_roots(complex(x[0], y[0]), m[0], kappa_s, gamma, ph)
        w = oracle.map_caustics(x, y, m, kappa_s, gamma, zc)
        wc = lm.chang_refsdal_caustic(complex(x[0], y[0]), m[0], kappa_s, gamma, ph)
        assert np.max(np.abs(w - wc)) < 1e-12


@pytest.mark.parametrize("n,seed,kappa_s,gamma", [(5, 11, 0.0, 0.3), (12, 12, 0.2, 0.6), (30, 13, 0.1, 0.05)])
def test_vieta_invariants_every_row(n, seed, kappa_s, gamma):
    """From P = c prod(z-z_i)^2 + sum m_i prod_{j!=i}(z-z_j)^2:
    sum_k z_k = 2 sum_i z_i and sum_k z_k^2 = 2 sum_i z_i^2 - 2 M / c."""
    x, y, m = _random_field(n, seed, mass="mixed")
    zs = x + 1j * y
    msteps = 40
    z, _, bad = oracle.critical_curves(x, y, m, kappa_s, gamma, msteps)
    assert bad == 0
    for j in range(msteps + 1):
        ph = oracle.phi(j, msteps)
        c = gamma - (1 - kappa_s) * np.exp(-1j * ph)
        s1 = z[j].sum()
        s2 = (z[j] ** 2).sum()
        scale = np.abs(z[j]).sum() + 1
        assert abs(s1 - 2 * zs.sum()) < 1e-11 * scale
        assert abs(s2 - (2 * (zs ** 2).sum() - 2 * m.sum() / c)) < 1e-11 * scale ** 2


@pytest.mark.parametrize("n,seed", [(1, 21), (2, 22), (4, 23), (6, 24)])
def test_tiny_fields_match_companion_roots(n, seed):
    """Brute force: roots of the explicitly formed polynomial (companion eigenvalues)."""
    x, y, m = _random_field(n, seed, spread=1.5, mass="mixed")
    for kappa_s, gamma in [(0.0, 0.25), (0.3, 0.45)]:
        for ph in [0.0, 1.1, math.pi, 4.0]:
            zo, left = oracle.solve_row(x, y, m, kappa_s, gamma, ph)
            assert left == 0
            zc = lm.companion_roots(x, y, m, kappa_s, gamma, ph)
            err, sep = lm.match_rows(zo, zc)
            assert len(zo) == 2 * n == len(zc)
            assert err < 1e-9 and err < 1e-3 * sep


def test_roots_count_and_distinct():
    f = synth.workload_small().fields[0]
    z, it, bad = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 100)
    assert bad == 0
    assert z.shape == (101, 2 * f.n)
    for j in range(0, 101, 10):
        assert oracle.min_separation(z[j]) > 1e-6
    # rows 0 and m (phi = 0 and 2 pi) hold the same set (Sec. 4.3)
    err, sep = lm.match_rows(z[0], z[-1])
    assert err < 1e-10


def test_critical_points_zero_lens_jacobian():
    """det of the lens map's Jacobian, by finite differences of w, vanishes at the roots of F
    (and the analytic 1/mu obeys the Appendix C bound from |F|)."""
    f = synth.workload_small().fields[0]
    z, _, _ = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 20)
    pts = z[::4].ravel()
    det = lm.jacobian_det_fd(f.x, f.y, f.m, f.kappa_s, f.gamma, pts)
    # scale: entries of the Jacobian are O(1 + |sum m/d^2|)
    for p, dv in zip(pts, det):
        j = 1.0 + abs(oracle.dF(f.x, f.y, f.m, p))
        assert abs(dv) < 1e-6 * j
    for j, row in enumerate(z[::4]):
        ph = oracle.phi(4 * j, 20)
        for p in row:
            Fa = abs(oracle.F(f.x, f.y, f.m, f.kappa_s, f.gamma, ph, p))
            bound = max(abs(Fa * Fa + 2 * Fa * (1 - f.kappa_s)), abs(Fa * Fa - 2 * Fa * (1 - f.kappa_s)))
            assert abs(oracle.inv_mu(f.x, f.y, f.m, f.kappa_s, f.gamma, p)) <= bound + 1e-13


def test_parametrisation_phase():
    """At a critical point, the lens-map derivatives satisfy dw/dz e^{i phi} = dw/dconj(z)
    (Sec. 3.1); checked with finite-difference Wirtinger derivatives of w."""
    f = synth.workload_small().fields[0]
    msteps = 16
    z, _, _ = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, msteps)
    h = 1e-6
    for j in range(0, msteps + 1, 3):
        ph = oracle.phi(j, msteps)
        for p in z[j][:6]:
            wx = (lm.lens_map(f.x, f.y, f.m, f.kappa_s, f.gamma, [p + h]) - lm.lens_map(f.x, f.y, f.m, f.kappa_s, f.gamma, [p - h]))[0] / (2 * h)
            wy = (lm.lens_map(f.x, f.y, f.m, f.kappa_s, f.gamma, [p + 1j * h]) - lm.lens_map(f.x, f.y, f.m, f.kappa_s, f.gamma, [p - 1j * h]))[0] / (2 * h)
            dwdz = 0.5 * (wx - 1j * wy)
            dwdzb = 0.5 * (wx + 1j * wy)
            assert abs(dwdz * np.exp(1j * ph) - dwdzb) < 1e-6 * (1 + abs(dwdzb))


@pytest.mark.parametrize("sep,loops", [(0.6, 3), (1.8, 1), (4.0, 2)])
def test_equal_mass_binary_topology(sep, loops):
    """Equal-mass binary without shear or smooth matter: close / intermediate / wide
    separations give 3 / 1 / 2 closed critical curves (transitions at 1/sqrt(2) and 2
    total-mass Einstein radii, i.e. 1 and 2 sqrt(2) unit-mass radii)."""
    x = np.array([-sep / 2, sep / 2])
    y = np.zeros(2)
    m = np.ones(2)
    z, _, bad = oracle.critical_curves(x, y, m, 0.0, 0.0, 200)
    assert bad == 0
    found, _ = lm.join_chains(z)
    assert len(found) == loops


def test_caustics_clockwise():
    """Caustics are traced clockwise (Sec. 5.1): each joined Chang-Refsdal caustic loop has
    negative signed area."""
    x, y, m = np.array([0.0]), np.array([0.0]), np.array([1.0])
    for kappa_s, gamma in [(0.0, 0.2), (0.2, 0.3)]:
        z, _, _ = oracle.critical_curves(x, y, m, kappa_s, gamma, 400)
        w = oracle.map_caustics(x, y, m, kappa_s, gamma, z)
        loops, _ = lm.join_chains(z)
        for lp in loops:
            assert lm.signed_area(lm.loop_polygon(w, lp)) < 0


def test_solve_row_cold_equals_warm_chain():
    """A cold start at phi_j finds the same root set as the warm-started chain row."""
    f = synth.workload_small().fields[0]
    z, _, _ = oracle.critical_curves(f.x, f.y, f.m, f.kappa_s, f.gamma, 50)
    for j in [0, 7, 33, 50]:
        zc, left = oracle.solve_row(f.x, f.y, f.m, f.kappa_s, f.gamma, oracle.phi(j, 50))
        assert left == 0
        err, sep = lm.match_rows(z[j], zc)
        assert err < 1e-11


def test_F_equals_lens_map_wirtinger_form():
    """F(z, phi) = conj(dw/dconj z) - conj(dw/dz) e^{-i phi} (Sec. 3.1 parametric form),
    with both Wirtinger derivatives of the lens map taken by finite differences."""
    f = synth.workload_small().fields[0]
    u = synth.uniform(31337, 3 * 20)
    h = 1e-6
    for t in range(20):
        p = complex(8 * (u[3 * t] - 0.5), 8 * (u[3 * t + 1] - 0.5))
        ph = 2 * math.pi * u[3 * t + 2]
        wx = (lm.lens_map(f.x, f.y, f.m, f.kappa_s, f.gamma, [p + h]) - lm.lens_map(f.x, f.y, f.m, f.kappa_s, f.gamma, [p - h]))[0] / (2 * h)
        wy = (lm.lens_map(f.x, f.y, f.m, f.kappa_s, f.gamma, [p + 1j * h]) - lm.lens_map(f.x, f.y, f.m, f.kappa_s, f.gamma, [p - 1j * h]))[0] / (2 * h)
        dwdz = 0.5 * (wx - 1j * wy)
        dwdzb = 0.5 * (wx + 1j * wy)
        ref = np.conj(dwdzb) - np.conj(dwdz) * np.exp(-1j * ph)
        got = oracle.F(f.x, f.y, f.m, f.kappa_s, f.gamma, ph, p)
        assert abs(got - ref) < 1e-6 * (1 + abs(ref))
        # dF/dz by central differences of F itself
        dref = (oracle.F(f.x, f.y, f.m, f.kappa_s, f.gamma, ph, p + h) - oracle.F(f.x, f.y, f.m, f.kappa_s, f.gamma, ph, p - h)) / (2 * h)
        assert abs(oracle.dF(f.x, f.y, f.m, p) - dref) < 1e-5 * (1 + abs(dref))


@pytest.mark.parametrize("kappa_s,gamma", [(0.0, 0.2), (0.3, 0.5), (0.0, 1.3)])
def test_newton_check_at_and_near_chang_refsdal_roots(kappa_s, gamma):
    """At the closed-form roots the Newton correction vanishes and w is the closed-form
    caustic; a root moved by delta gets a correction of length |delta| (to first order), so a
    wrong factor in F' or a wrong phase row would show."""
    x, y, m = np.array([0.7]), np.array([-0.4]), np.array([0.6])
    msteps, row0 = 64, 5
    rows = [lm.chang_refsdal_roots(complex(x[0], y[0]), m[0], kappa_s, gamma, oracle.phi(row0 + r, msteps))
            for r in range(4)]
    z = np.array(rows)
    step, w = oracle.newton_check(x, y, m, kappa_s, gamma, msteps, z, row0=row0)
    assert step.max() < 1e-13
    for r in range(4):
        wc = lm.chang_refsdal_caustic(complex(x[0], y[0]), m[0], kappa_s, gamma, oracle.phi(row0 + r, msteps))
        assert np.abs(w[r] - wc).max() < 1e-12
    delta = 1e-6 * np.exp(1j * np.array([[0.3, 2.0], [4.1, 1.1], [5.5, 0.2], [3.3, 2.8]]))
    step2, _ = oracle.newton_check(x, y, m, kappa_s, gamma, msteps, z + delta, row0=row0)
    assert np.abs(step2 / np.abs(delta) - 1).max() < 1e-4
    # the same points attributed to other rows are not roots there
    step3, _ = oracle.newton_check(x, y, m, kappa_s, gamma, msteps, z, row0=row0 + 1)
    assert step3.min() > 1e-4


def test_newton_check_matches_oracle_sums_on_a_field():
    """On a random 25-star field the per-point values equal the oracle's own F, F' and lens
    map (written separately, with complex division) at every point and phase row."""
    x, y, m = _random_field(25, 31, mass="var")
    kappa_s, gamma, msteps, row0 = 0.15, 0.45, 40, 7
    u = synth.uniform(32, 2 * 3 * 6)
    z = ((u[0::2] - 0.5) * 8 + 1j * (u[1::2] - 0.5) * 8).reshape(3, 6)
    step, w = oracle.newton_check(x, y, m, kappa_s, gamma, msteps, z, row0=row0)
    wo = oracle.map_caustics(x, y, m, kappa_s, gamma, z)
    assert np.abs(w - wo).max() < 1e-12 * (1 + np.abs(wo).max())
    for r in range(3):
        for k in range(6):
            F = oracle.F(x, y, m, kappa_s, gamma, oracle.phi(row0 + r, msteps), z[r, k])
            dF = oracle.dF(x, y, m, z[r, k])
            assert abs(step[r, k] - abs(F) / abs(dF)) < 1e-12 * step[r, k]
