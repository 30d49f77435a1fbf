"""Pins of the oracle's rectangular microlens field (Sec. 4.2, Appendices A and B).

Each test checks the oracle against something other than itself:
- alpha_s against its definition, the deflection of a uniform rectangular sheet
  (numerical quadrature), and against the Appendix B error bound of its truncation;
- the final form of dalpha_s/dconj(z) against finite differences of alpha_s, and F, F'
  against finite differences of the lens map w (the parametric critical-curve condition);
- the Aberth roots against companion-matrix roots of P = F prod (z - z_i)^2, whose
  coefficients are sampled by FFT (n_r = 2N + t - 1 roots);
- det J = 0 at the roots; the truncation-order rule; the kappa_* = 0 limit.
"""
import cmath
import math

import numpy as np
import pytest

import oracle

integrate = pytest.importorskip("scipy.integrate")


def field(n, c1, c2, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-c1, c1, n), rng.uniform(-c2, c2, n), rng.uniform(0.2, 1.0, n)


def alpha_quadrature(kst, c1, c2, z):
    """-(kappa_*/pi) int int dA' / conj(z - z') over the rectangle, split at z."""
    fr = lambda y, x: (1.0 / np.conj(z - (x + 1j * y))).real
    fi = lambda y, x: (1.0 / np.conj(z - (x + 1j * y))).imag
    xs, ys = [-c1, z.real, c1], [-c2, z.imag, c2]
    tot = 0j
    for i in range(2):
        for k in range(2):
            kw = dict(epsabs=1e-11, epsrel=1e-11)
            tot += integrate.dblquad(fr, xs[i], xs[i + 1], ys[k], ys[k + 1], **kw)[0]
            tot += 1j * integrate.dblquad(fi, xs[i], xs[i + 1], ys[k], ys[k + 1], **kw)[0]
    return -(kst / math.pi) * tot


@pytest.mark.parametrize("z", [0.3 + 0.2j, -1.1 + 0.7j, 2.0 - 1.5j])
def test_alpha_exact_is_the_sheet_deflection(z):
    kst, c1, c2 = 0.4, 3.0, 2.0
    a = oracle.rect_alpha(kst, c1, c2, z, t=-1)
    # the sheet is extended to infinity outside the rectangle (Appendix B): inside it the
    # closed form is the finite rectangle's deflection
    assert abs(a - alpha_quadrature(kst, c1, c2, z)) < 1e-9


@pytest.mark.parametrize("t", [5, 9, 15])
@pytest.mark.parametrize("s", [1.5, 2.0, 3.0])
def test_truncation_within_appendix_b_bound(t, s):
    kst, c1, c2 = 0.3, 4.0, 2.5
    ac = math.hypot(c1, c2)
    bound = (kst / math.pi) * (4.0 / (t + 1)) * s ** -(t + 1) * ac * (s + 1) / (s - 1)
    worst = 0.0
    for k in range(24):
        z = ac / s * cmath.exp(1j * (2 * math.pi * k / 24 + 0.1))
        worst = max(worst, abs(oracle.rect_alpha(kst, c1, c2, z, t) - oracle.rect_alpha(kst, c1, c2, z, -1)))
    assert worst <= bound
    assert worst > 1e-3 * bound  # the bound is not vacuous here


@pytest.mark.parametrize("t", [3, 7, 11])
@pytest.mark.parametrize("z", [0.4 + 0.3j, -2.0 + 1.1j, 3.5 - 2.5j])
def test_final_form_is_derivative_of_truncated_alpha(t, z):
    kst, c1, c2 = 0.45, 3.0, 2.2
    h = 1e-5
    a = lambda u: oracle.rect_alpha(kst, c1, c2, u, t)
    d_dzb = ((a(z + h) - a(z - h)) + 1j * (a(z + 1j * h) - a(z - 1j * h))) / (4 * h)
    d_dz = ((a(z + h) - a(z - h)) - 1j * (a(z + 1j * h) - a(z - 1j * h))) / (4 * h)
    assert abs(d_dzb - oracle.rect_dalpha_dzb(kst, c1, c2, t, z)) < 1e-8
    assert abs(d_dz - (-kst)) < 1e-8  # dalpha_s/dz = -kappa_* (Appendix B)


@pytest.mark.parametrize("phi", [0.3, 2.0, 4.4])
def test_F_is_the_parametric_condition_of_w(phi):
    x, y, m = field(5, 3.0, 2.0, 1)
    ks, g, R = 0.1, 0.3, oracle.Rect(0.35, 3.0, 2.0, 9)
    h = 1e-5
    for z in [0.7 + 0.9j, -2.1 - 0.4j, 1.3 - 1.7j]:
        w = lambda u: oracle.map_caustics(x, y, m, ks, g, np.array([u]), rect=R)[0]
        dwdz = ((w(z + h) - w(z - h)) - 1j * (w(z + 1j * h) - w(z - 1j * h))) / (4 * h)
        dwdzb = ((w(z + h) - w(z - h)) + 1j * (w(z + 1j * h) - w(z - 1j * h))) / (4 * h)
        # Sec. 3.1: dw/dz e^{i phi} - dw/dconj(z) = 0, conjugated and negated
        expect = np.conj(dwdzb) - np.conj(dwdz) * cmath.exp(-1j * phi)
        got = oracle.F(x, y, m, ks, g, phi, z, rect=R)
        assert abs(got - expect) < 1e-7 * (1 + abs(got))
        Fz = lambda u: oracle.F(x, y, m, ks, g, phi, u, rect=R)
        dF_fd = (Fz(z + h) - Fz(z - h)) / (2 * h)
        assert abs(oracle.dF(x, y, m, z, rect=R) - dF_fd) < 1e-6 * (1 + abs(dF_fd))


def companion_roots(x, y, m, ks, g, phi, R):
    """Roots of P(z) = F(z) prod (z - z_i)^2, a polynomial of degree 2N + t - 1, from its
    coefficients sampled by FFT on a circle (numpy's companion-matrix eigenvalues)."""
    n = len(x)
    deg = 2 * n + R.t - 1
    M = 2 * (deg + 1) + 8
    rad = 1.3 * max(math.hypot(R.c1, R.c2), 1.0)
    zs = rad * np.exp(2j * np.pi * np.arange(M) / M)
    zi = x + 1j * y
    vals = np.array([oracle.F(x, y, m, ks, g, phi, u, rect=R) * np.prod((u - zi) ** 2) for u in zs])
    coef = np.fft.fft(vals) / M / rad ** np.arange(M)  # coef[k] of z^k
    assert np.abs(coef[deg + 1:M - 1]).max() < 1e-9 * np.abs(coef[deg])  # degree is exactly deg
    return np.roots(coef[:deg + 1][::-1])


@pytest.mark.parametrize("n,t", [(1, 5), (2, 7), (3, 9)])
def test_roots_match_companion_matrix(n, t):
    x, y, m = field(n, 2.5, 1.8, 10 + n)
    ks, g, R = 0.05, 0.25, oracle.Rect(0.3, 2.5, 1.8, t)
    for phi in [0.0, 1.1, 3.0]:
        z, left = oracle.solve_row(x, y, m, ks, g, phi, rect=R)
        assert left == 0 and len(z) == R.n_roots(n) == 2 * n + t - 1
        ref = companion_roots(x, y, m, ks, g, phi, R)
        d = np.abs(z[:, None] - ref[None, :])
        assert len(set(d.argmin(axis=1).tolist())) == len(z)  # one-to-one
        assert d.min(axis=1).max() < 1e-7


def test_det_J_vanishes_at_roots_and_roots_are_distinct():
    x, y, m = field(12, 4.0, 3.0, 5)
    ks, g = 0.0, 0.35
    t = oracle.rect_choose_t(0.4, 4.0, 3.0)
    R = oracle.Rect(0.4, 4.0, 3.0, t)
    z, left = oracle.solve_row(x, y, m, ks, g, 2.2, rect=R)
    assert left == 0 and len(z) == 24 + t - 1
    assert oracle.min_separation(z) > 1e-3
    h = 1e-6
    for u in z[::3]:
        w = lambda v: oracle.map_caustics(x, y, m, ks, g, np.array([v]), rect=R)[0]
        a = ((w(u + h) - w(u - h)) - 1j * (w(u + 1j * h) - w(u - 1j * h))) / (4 * h)
        b = ((w(u + h) - w(u - h)) + 1j * (w(u + 1j * h) - w(u - 1j * h))) / (4 * h)
        assert abs(abs(a) ** 2 - abs(b) ** 2) < 1e-5 * (1 + abs(b) ** 2)


@pytest.mark.parametrize("c1,c2", [(3.0, 3.0), (5.0, 2.0), (2.0, 6.0), (40.0, 40.0)])
@pytest.mark.parametrize("eps,s", [(1e-9, 2.0), (1e-6, 1.5)])
def test_truncation_order_rule(c1, c2, eps, s):
    kst = 0.4
    ac, th = math.hypot(c1, c2), math.atan2(c2, c1)

    def ok(t):
        b = (kst / math.pi) * (4.0 / (t + 1)) * s ** -(t + 1) * ac * (s + 1) / (s - 1)
        r = math.fmod((t - 1) * th, math.pi)
        return b <= eps and 0.1 * math.pi < r < 0.9 * math.pi

    t = oracle.rect_choose_t(kst, c1, c2, eps, s)
    assert t % 2 == 1 and ok(t)
    assert not any(ok(u) for u in range(3, t, 2))
    if c1 == c2:  # square: (t - 1) pi/4 must not be a multiple of pi
        assert (t - 1) % 4 == 2


def test_zero_sheet_is_the_disc_model():
    x, y, m = field(6, 3.0, 2.0, 7)
    R = oracle.Rect(0.0, 3.0, 2.0, 9)
    for z in [0.5 + 0.5j, -1.5 + 0.2j]:
        assert abs(oracle.F(x, y, m, 0.2, 0.3, 1.0, z, rect=R) - oracle.F(x, y, m, 0.2, 0.3, 1.0, z)) < 1e-14
        a = oracle.map_caustics(x, y, m, 0.2, 0.3, np.array([z]), rect=R)[0]
        b = oracle.map_caustics(x, y, m, 0.2, 0.3, np.array([z]))[0]
        assert abs(a - b) < 1e-13


def test_chain_matrix_rect():
    x, y, m = field(8, 3.0, 2.0, 9)
    t = oracle.rect_choose_t(0.3, 3.0, 2.0)
    R = oracle.Rect(0.3, 3.0, 2.0, t)
    z, it, bad = oracle.critical_curves(x, y, m, 0.0, 0.3, 32, rect=R)
    assert bad == 0 and z.shape == (33, 16 + t - 1)
    for j in range(0, 33, 8):
        phi = oracle.phi(j, 32)
        assert max(abs(oracle.F(x, y, m, 0.0, 0.3, phi, u, rect=R)) for u in z[j]) < 1e-11


@pytest.mark.parametrize("theta,t_bad", [(math.pi / 4, 9), (math.pi / 4 - 0.01, 9), (math.pi / 4 + 0.01, 9),
                                         (math.pi / 3, 7)])
def test_truncation_order_skips_vanishing_leading_term(theta, t_bad):
    """eps chosen so that the bound alone would give t_bad, whose (t_bad - 1) Arg c lies
    within 10% of pi of a multiple of pi: the rule must move on to a larger odd t."""
    kst, s, ac = 0.4, 2.0, 5.0
    c1, c2 = ac * math.cos(theta), ac * math.sin(theta)
    bound = lambda t: (kst / math.pi) * (4.0 / (t + 1)) * s ** -(t + 1) * ac * (s + 1) / (s - 1)
    eps = bound(t_bad) * 1.0001
    r = math.fmod((t_bad - 1) * theta, math.pi)
    assert not (0.1 * math.pi < r < 0.9 * math.pi)
    t = oracle.rect_choose_t(kst, c1, c2, eps, s)
    assert t > t_bad and t % 2 == 1
    rt = math.fmod((t - 1) * theta, math.pi)
    assert 0.1 * math.pi < rt < 0.9 * math.pi
