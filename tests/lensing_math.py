"""Independent closed forms and brute-force helpers used to pin the oracle.

Nothing here calls the oracle or the CUDA path.  Each helper states the mathematics it
writes out.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def chang_refsdal_roots(z0: complex, mass: float, kappa_s: float, gamma: float, phi: float):
    """One point mass with shear and smooth matter: F = 0 gives
    (z - z0)^2 = m / ((1 - kappa_s) e^{-i phi} - gamma), so z = z0 +- sqrt(...)."""
    q = (1.0 - kappa_s) * np.exp(-1j * phi) - gamma
    r = np.sqrt(mass / q)
    return np.array([z0 + r, z0 - r])


def chang_refsdal_caustic(z0: complex, mass: float, kappa_s: float, gamma: float, phi: float):
    """Caustic point of each Chang-Refsdal critical point.  With d = z - z0,
    d^2 = m/q and |d|^2 = m/|q|, so m / conj(d) = d |q| and the lens map becomes
    w = z0-image + (1 - kappa_s - |q|) d + gamma conj(d) with the constant part
    (1 - kappa_s) z0 + gamma conj(z0)."""
    q = (1.0 - kappa_s) * np.exp(-1j * phi) - gamma
    d = np.sqrt(mass / q)
    ds = np.array([d, -d])
    base = (1.0 - kappa_s) * z0 + gamma * np.conj(z0)
    return base + (1.0 - kappa_s - abs(q)) * ds + gamma * np.conj(ds)


def rationalised_poly(xs, ys, ms, kappa_s, gamma, phi):
    """Coefficients (highest first) of P(z) = F(z) prod_i (z - z_i)^2
    = c prod_j (z - z_j)^2 + sum_i m_i prod_{j != i} (z - z_j)^2, c = gamma - (1-kappa_s) e^{-i phi}."""
    zs = np.asarray(xs) + 1j * np.asarray(ys)
    c = gamma - (1.0 - kappa_s) * np.exp(-1j * phi)
    full = np.array([1.0 + 0j])
    for zi in zs:
        full = np.polymul(full, [1.0, -2 * zi, zi * zi])
    p = c * full
    for i, mi in enumerate(ms):
        part = np.array([1.0 + 0j])
        for j, zj in enumerate(zs):
            if j != i:
                part = np.polymul(part, [1.0, -2 * zj, zj * zj])
        p = np.polyadd(p, mi * part)
    return p


def companion_roots(xs, ys, ms, kappa_s, gamma, phi):
    """Roots of the rationalised polynomial by companion-matrix eigenvalues (numpy.roots),
    each refined by Newton steps on the polynomial itself."""
    p = rationalised_poly(xs, ys, ms, kappa_s, gamma, phi)
    r = np.roots(p)
    dp = np.polyder(p)
    for _ in range(5):
        r = r - np.polyval(p, r) / np.polyval(dp, r)
    return r


def lens_map(xs, ys, ms, kappa_s, gamma, z):
    """w = (1 - kappa_s) z + gamma conj(z) - sum m_i / conj(z - z_i) (numpy, vectorised)."""
    z = np.asarray(z, dtype=np.complex128)
    zs = np.asarray(xs) + 1j * np.asarray(ys)
    s = np.zeros_like(z)
    for zi, mi in zip(zs, ms):
        s = s + mi / np.conj(z - zi)
    return (1.0 - kappa_s) * z + gamma * np.conj(z) - s


def jacobian_det_fd(xs, ys, ms, kappa_s, gamma, z, h=1e-5):
    """det of the real 2x2 Jacobian of the lens map by central differences."""
    z = np.asarray(z, dtype=np.complex128)
    wx = (lens_map(xs, ys, ms, kappa_s, gamma, z + h) - lens_map(xs, ys, ms, kappa_s, gamma, z - h)) / (2 * h)
    wy = (lens_map(xs, ys, ms, kappa_s, gamma, z + 1j * h) - lens_map(xs, ys, ms, kappa_s, gamma, z - 1j * h)) / (2 * h)
    return wx.real * wy.imag - wx.imag * wy.real


def image_count(xs, ys, ms, kappa_s, gamma, w, tol=1e-7):
    """Number of images of a point source at w: roots of the lens-equation polynomial
    obtained by eliminating conj(z) (conjugate equation solved for conj(z) and substituted
    back), kept only where the lens equation itself holds."""
    a = 1.0 - kappa_s
    zs = [complex(x, y) for x, y in zip(xs, ys)]
    n = len(zs)

    def lin(c0, c1):  # c1 z + c0 -> highest-first
        return np.array([c1, c0], dtype=np.complex128)

    pi_all = np.array([1.0 + 0j])
    for zi in zs:
        pi_all = np.polymul(pi_all, lin(-zi, 1.0))
    pi_ex = []
    for i in range(n):
        p = np.array([1.0 + 0j])
        for j, zj in enumerate(zs):
            if j != i:
                p = np.polymul(p, lin(-zj, 1.0))
        pi_ex.append(p)
    rd = a * pi_all
    rn = np.polymul(lin(np.conj(w), -gamma), pi_all)
    for i in range(n):
        rn = np.polyadd(rn, ms[i] * pi_ex[i])
    qs = [np.polysub(rn, np.conj(zs[i]) * rd) for i in range(n)]
    prod_q = np.array([1.0 + 0j])
    for q in qs:
        prod_q = np.polymul(prod_q, q)
    poly = np.polymul(np.polymul(lin(w, -a), rd), prod_q)
    poly = np.polysub(poly, gamma * np.polymul(rn, prod_q))
    for i in range(n):
        others = np.array([1.0 + 0j])
        for j in range(n):
            if j != i:
                others = np.polymul(others, qs[j])
        poly = np.polyadd(poly, ms[i] * np.polymul(np.polymul(rd, rd), others))
    # strip leading ~zeros
    scale = np.abs(poly).max()
    k = 0
    while k < len(poly) - 1 and abs(poly[k]) < 1e-14 * scale:
        k += 1
    poly = poly[k:]
    cand = np.roots(poly)
    dp = np.polyder(poly)
    for _ in range(3):
        cand = cand - np.polyval(poly, cand) / np.polyval(dp, cand)
    good = []
    for zc in cand:
        if not np.isfinite(zc):
            continue
        if abs(lens_map(xs, ys, ms, kappa_s, gamma, np.array([zc]))[0] - w) < tol:
            if all(abs(zc - g) > 1e-6 for g in good):
                good.append(zc)
    return len(good)


def orient_exact(ax, ay, bx, by, cx, cy) -> int:
    """Sign of (a - c) x (b - c) in exact rational arithmetic."""
    A = [Fraction(v) for v in (ax, ay, bx, by, cx, cy)]
    det = (A[0] - A[4]) * (A[3] - A[5]) - (A[1] - A[5]) * (A[2] - A[4])
    return (det > 0) - (det < 0)


def match_rows(a, b):
    """Greedy nearest-neighbour matching of two root multisets; returns max distance and
    the smallest separation inside a (so the caller can require an unambiguous match)."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.abs(a[:, None] - b[None, :])
    used = np.zeros(len(b), dtype=bool)
    worst = 0.0
    for i in np.argsort(d.min(axis=1)):
        order = np.argsort(d[i])
        for j in order:
            if not used[j]:
                used[j] = True
                worst = max(worst, d[i, j])
                break
    sep = np.abs(a[:, None] - a[None, :])
    np.fill_diagonal(sep, np.inf)
    return worst, float(sep.min())


def join_chains(z):
    """Join chains (columns of the (m+1) x n_r matrix) into closed loops: the end of
    chain k (row m) is the start (row 0) of chain sigma(k).  Returns the list of loops,
    each a list of chain indices."""
    end = z[-1]
    start = z[0]
    sigma = [int(np.argmin(np.abs(start - e))) for e in end]
    seen = [False] * len(sigma)
    loops = []
    for k in range(len(sigma)):
        if seen[k]:
            continue
        loop = []
        j = k
        while not seen[j]:
            seen[j] = True
            loop.append(j)
            j = sigma[j]
        loops.append(loop)
    return loops, sigma


def loop_polygon(z, loop):
    """Concatenate the chains of one loop into one closed polyline (rows 0..m-1 each)."""
    pts = []
    for k in loop:
        pts.extend(list(z[:-1, k]))
    return np.array(pts)


def signed_area(poly):
    x = poly.real
    y = poly.imag
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))
