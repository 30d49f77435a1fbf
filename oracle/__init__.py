"""Plain FP64 CPU oracle for microlensing critical curves and caustics.

TEST INFRASTRUCTURE ONLY.  The slow, obviously-correct reference that the CUDA path is
checked against (Weisenbach 2025, Secs. 3-5 and Appendices A and C).  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA library and never imports the product package.

The arithmetic lives in ``cc_oracle.c`` (C99, FP64, ``-ffp-contract=off``); this module
compiles it with gcc and wraps it with ctypes.  Parity status of each function is in the
C file's comments; everything here is pinned by tests in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_DP = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)
_U8P = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_liboracle.so`` (OpenMP if gcc supports it)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base + ["-o", tmp, _SRC, "-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, dbl, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int32
        lib.orc_F.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, dbl, _DP, _DP]
        lib.orc_F.restype = dbl
        lib.orc_dF.argtypes = [_DP, _DP, _DP, i64, _DP, _DP]
        lib.orc_dF.restype = dbl
        lib.orc_inv_mu.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, _DP]
        lib.orc_inv_mu.restype = dbl
        lib.orc_solve_row.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, dbl, _DP, _DP, ctypes.c_int, dbl, _I32P]
        lib.orc_solve_row.restype = i64
        lib.orc_phi.argtypes = [i64, i64]
        lib.orc_phi.restype = dbl
        lib.orc_critical_curves.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, i64, dbl, ctypes.c_int,
                                            ctypes.c_int, _DP, _I32P]
        lib.orc_critical_curves.restype = i64
        lib.orc_map_caustics.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, _DP, i64, _DP]
        lib.orc_map_caustics.restype = None
        lib.orc_min_separation.argtypes = [_DP, i64]
        lib.orc_min_separation.restype = dbl
        lib.orc_orient2d.argtypes = [dbl] * 6
        lib.orc_orient2d.restype = ctypes.c_int
        lib.orc_pixel_center.argtypes = [dbl, dbl, i32, i32]
        lib.orc_pixel_center.restype = dbl
        lib.orc_winding_at.argtypes = [_DP, i64, i64, dbl, dbl]
        lib.orc_winding_at.restype = i64
        lib.orc_crossing_map.argtypes = [_DP, i64, i64, dbl, dbl, dbl, dbl, i32, i32, _I32P]
        lib.orc_crossing_map.restype = None
        lib.orc_crossing_rows.argtypes = [_DP, i64, i64, dbl, dbl, dbl, dbl, i32, i32, _I32P, i32, _I32P]
        lib.orc_crossing_rows.restype = None
        lib.orc_newton_check.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, i64, i64, i64, i64, _DP, _DP, _DP]
        lib.orc_newton_check.restype = None
        lib.orc_feature_mask.argtypes = [_I32P, i32, i32, _U8P]
        lib.orc_feature_mask.restype = None
        lib.orc_distance_map_brute.argtypes = [_I32P, i32, i32, dbl, _DP]
        lib.orc_distance_map_brute.restype = None
        lib.orc_distance_map_separable.argtypes = [_I32P, i32, i32, dbl, _DP]
        lib.orc_distance_map_separable.restype = None
        lib.orc_moving_distance_map.argtypes = [_I32P, i32, i32, dbl, dbl, _DP]
        lib.orc_moving_distance_map.restype = None
        ci = ctypes.c_int
        lib.orc_rect_F.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, dbl, dbl, dbl, ci, dbl, _DP, _DP]
        lib.orc_rect_F.restype = dbl
        lib.orc_rect_dF.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, dbl, ci, _DP, _DP]
        lib.orc_rect_dF.restype = dbl
        lib.orc_rect_alpha.argtypes = [dbl, dbl, dbl, ci, _DP, _DP]
        lib.orc_rect_alpha.restype = None
        lib.orc_rect_dalpha_dzb.argtypes = [dbl, dbl, dbl, ci, _DP, _DP]
        lib.orc_rect_dalpha_dzb.restype = None
        lib.orc_rect_choose_t.argtypes = [dbl, dbl, dbl, dbl, dbl]
        lib.orc_rect_choose_t.restype = ci
        lib.orc_rect_solve_row.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, dbl, dbl, dbl, ci, dbl, _DP, _DP, ci,
                                           dbl, _I32P]
        lib.orc_rect_solve_row.restype = i64
        lib.orc_rect_critical_curves.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, dbl, dbl, dbl, ci, i64, dbl, ci,
                                                 ci, _DP, _I32P]
        lib.orc_rect_critical_curves.restype = i64
        lib.orc_rect_map_caustics.argtypes = [_DP, _DP, _DP, i64, dbl, dbl, dbl, dbl, dbl, ci, _DP, i64, _DP]
        lib.orc_rect_map_caustics.restype = None
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        lib.orc_set_num_threads.restype = None
        _lib = lib
        return lib


def _d(a):
    return a.ctypes.data_as(_DP)


def _stars(x, y, m):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    if not (x.shape == y.shape == m.shape and x.ndim == 1):
        raise ValueError("x, y, m must be 1-D arrays of equal length")
    return x, y, m


class Rect:
    """Rectangular microlens field (Sec. 4.2, Appendix B): smooth sheet of convergence
    kappa_star, corner c = c1 + i c2, logarithm series truncated at the odd order t."""

    def __init__(self, kappa_star: float, c1: float, c2: float, t: int):
        if t < 1 or t % 2 == 0:
            raise ValueError("t must be odd and >= 1")
        self.kappa_star, self.c1, self.c2, self.t = float(kappa_star), float(c1), float(c2), int(t)

    def n_roots(self, n: int) -> int:
        return 2 * n + self.t - 1

    def args(self):
        return self.kappa_star, self.c1, self.c2, self.t


def rect_choose_t(kappa_star, c1, c2, eps=1e-9, s=2.0) -> int:
    """Odd truncation order from the Appendix B error bound, moved away from orders whose
    leading coefficient vanishes ((t - 1) Arg c a multiple of pi)."""
    return int(_load().orc_rect_choose_t(float(kappa_star), float(c1), float(c2), float(eps), float(s)))


def rect_alpha(kappa_star, c1, c2, z, t=-1):
    """alpha_s(z) of the rectangle (Appendix B); t < 0: exact logarithms."""
    zz = np.array([complex(z).real, complex(z).imag])
    out = np.zeros(2)
    _load().orc_rect_alpha(float(kappa_star), float(c1), float(c2), int(t), _d(zz), _d(out))
    return complex(out[0], out[1])


def rect_dalpha_dzb(kappa_star, c1, c2, t, z):
    """dalpha_s/dconj(z) of the rectangle at z (Appendix B, final form)."""
    zz = np.array([complex(z).real, complex(z).imag])
    out = np.zeros(2)
    _load().orc_rect_dalpha_dzb(float(kappa_star), float(c1), float(c2), int(t), _d(zz), _d(out))
    return complex(out[0], out[1])


def num_threads() -> int:
    """OpenMP threads the oracle uses (1 when built without OpenMP)."""
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (for timing runs)."""
    _load().orc_set_num_threads(int(n))


def phi(j: int, msteps: int) -> float:
    """phi_j = 2 pi j / m, computed exactly as the oracle does (Sec. 4.3)."""
    return float(_load().orc_phi(int(j), int(msteps)))


def F(x, y, m, kappa_s, gamma, phi_, z, rect: Rect | None = None):
    """F(z, phi) of the parametric critical-curve equation (Sec. 3.1, Appendix A; with
    rect, the rectangular field of Appendix B)."""
    x, y, m = _stars(x, y, m)
    zz = np.array([complex(z).real, complex(z).imag])
    out = np.zeros(2)
    if rect is None:
        _load().orc_F(_d(x), _d(y), _d(m), len(x), kappa_s, gamma, phi_, _d(zz), _d(out))
    else:
        _load().orc_rect_F(_d(x), _d(y), _d(m), len(x), kappa_s, gamma, *rect.args(), phi_, _d(zz), _d(out))
    return complex(out[0], out[1])


def dF(x, y, m, z, rect: Rect | None = None):
    """dF/dz = -2 sum m_i/(z - z_i)^3 (minus the rectangle's polynomial derivative)."""
    x, y, m = _stars(x, y, m)
    zz = np.array([complex(z).real, complex(z).imag])
    out = np.zeros(2)
    if rect is None:
        _load().orc_dF(_d(x), _d(y), _d(m), len(x), _d(zz), _d(out))
    else:
        _load().orc_rect_dF(_d(x), _d(y), _d(m), len(x), *rect.args(), _d(zz), _d(out))
    return complex(out[0], out[1])


def inv_mu(x, y, m, kappa_s, gamma, z):
    """1/mu = det J at z (Sec. 2.1, Appendix C)."""
    x, y, m = _stars(x, y, m)
    zz = np.array([complex(z).real, complex(z).imag])
    return float(_load().orc_inv_mu(_d(x), _d(y), _d(m), len(x), kappa_s, gamma, _d(zz)))


def solve_row(x, y, m, kappa_s, gamma, phi_, z0=None, max_iter=500, tol=1e-9, return_iters=False,
              rect: Rect | None = None):
    """Roots of F(., phi) for one row: Jacobi Aberth (from z0, or from the initial guesses
    when z0 is None) followed by a Newton polish.  Returns (z[n_r] complex128, unfrozen);
    n_r = 2N, or 2N + t - 1 for a rectangular field."""
    x, y, m = _stars(x, y, m)
    n = len(x)
    nr = 2 * n if rect is None else rect.n_roots(n)
    out = np.zeros(nr, dtype=np.complex128)
    zin = None
    if z0 is not None:
        zin = np.ascontiguousarray(z0, dtype=np.complex128)
        if zin.shape != (nr,):
            raise ValueError("z0 must have n_r entries")
    iters = np.zeros(nr, dtype=np.int32)
    zp = None if zin is None else zin.view(np.float64).ctypes.data_as(_DP)
    if rect is None:
        left = _load().orc_solve_row(_d(x), _d(y), _d(m), n, kappa_s, gamma, phi_, zp,
                                     out.view(np.float64).ctypes.data_as(_DP), int(max_iter), tol,
                                     iters.ctypes.data_as(_I32P))
    else:
        left = _load().orc_rect_solve_row(_d(x), _d(y), _d(m), n, kappa_s, gamma, *rect.args(), phi_, zp,
                                          out.view(np.float64).ctypes.data_as(_DP), int(max_iter), tol,
                                          iters.ctypes.data_as(_I32P))
    if return_iters:
        return out, int(left), iters
    return out, int(left)


def critical_curves(x, y, m, kappa_s, gamma, msteps, tol=1e-9, max_iter_cold=500, max_iter_warm=200,
                    rect: Rect | None = None):
    """Chain matrix of Sec. 4.3: (m+1) x n_r complex128 roots, row j at phi_j = 2 pi j/m.
    Returns (z, iters, unfrozen_total)."""
    if msteps < 2 or msteps % 2:
        raise ValueError("m must be even and >= 2")
    x, y, m = _stars(x, y, m)
    n = len(x)
    nr = 2 * n if rect is None else rect.n_roots(n)
    z = np.zeros((msteps + 1, nr), dtype=np.complex128)
    it = np.zeros((msteps + 1, nr), dtype=np.int32)
    zp, ip = z.view(np.float64).ctypes.data_as(_DP), it.ctypes.data_as(_I32P)
    if rect is None:
        bad = _load().orc_critical_curves(_d(x), _d(y), _d(m), n, kappa_s, gamma, int(msteps), tol,
                                          int(max_iter_cold), int(max_iter_warm), zp, ip)
    else:
        bad = _load().orc_rect_critical_curves(_d(x), _d(y), _d(m), n, kappa_s, gamma, *rect.args(), int(msteps),
                                               tol, int(max_iter_cold), int(max_iter_warm), zp, ip)
    return z, it, int(bad)


def map_caustics(x, y, m, kappa_s, gamma, z, rect: Rect | None = None):
    """Lens map w(z) of every critical point (Sec. 3.1; with rect, alpha_s of Appendix B);
    same shape as z."""
    x, y, m = _stars(x, y, m)
    zz = np.ascontiguousarray(z, dtype=np.complex128)
    w = np.zeros_like(zz)
    zp, wp = zz.view(np.float64).ctypes.data_as(_DP), w.view(np.float64).ctypes.data_as(_DP)
    if rect is None:
        _load().orc_map_caustics(_d(x), _d(y), _d(m), len(x), kappa_s, gamma, zp, zz.size, wp)
    else:
        _load().orc_rect_map_caustics(_d(x), _d(y), _d(m), len(x), kappa_s, gamma, *rect.args(), zp, zz.size, wp)
    return w


def min_separation(zrow):
    zz = np.ascontiguousarray(zrow, dtype=np.complex128)
    return float(_load().orc_min_separation(zz.view(np.float64).ctypes.data_as(_DP), zz.size))


def orient2d(ax, ay, bx, by, cx, cy) -> int:
    """Exact sign of (a-c) x (b-c): +1 if c is left of a->b, -1 right, 0 collinear."""
    return int(_load().orc_orient2d(float(ax), float(ay), float(bx), float(by), float(cx), float(cy)))


def pixel_center(lo, hi, cnt, i) -> float:
    return float(_load().orc_pixel_center(float(lo), float(hi), int(cnt), int(i)))


def winding_at(w, px, py) -> int:
    """Sunday winding number of the caustic polygons (columns of w) around (px, py)."""
    ww = np.ascontiguousarray(w, dtype=np.complex128)
    rows, nr = ww.shape
    return int(_load().orc_winding_at(ww.view(np.float64).ctypes.data_as(_DP), rows, nr, px, py))


def crossing_map(w, x0, x1, y0, y1, W, H):
    """N_cc = -winding number at every pixel centre (Sec. 5.1); int32 [H, W]."""
    ww = np.ascontiguousarray(w, dtype=np.complex128)
    rows, nr = ww.shape
    out = np.zeros((H, W), dtype=np.int32)
    _load().orc_crossing_map(ww.view(np.float64).ctypes.data_as(_DP), rows, nr, x0, x1, y0, y1,
                             int(W), int(H), out.ctypes.data_as(_I32P))
    return out


def crossing_rows(w, x0, x1, y0, y1, W, H, rows):
    """The listed pixel rows of crossing_map(w, x0, x1, y0, y1, W, H): the same pixel
    centres and decisions, int32 [len(rows), W]."""
    rl = np.ascontiguousarray(rows, dtype=np.int32)
    if rl.ndim != 1 or (rl.size and (rl.min() < 0 or rl.max() >= H)):
        raise ValueError("rows must be indices in [0, H)")
    ww = np.ascontiguousarray(w, dtype=np.complex128)
    nrows, nr = ww.shape
    out = np.zeros((rl.size, W), dtype=np.int32)
    _load().orc_crossing_rows(ww.view(np.float64).ctypes.data_as(_DP), nrows, nr, x0, x1, y0, y1,
                              int(W), int(H), rl.ctypes.data_as(_I32P), int(rl.size), out.ctypes.data_as(_I32P))
    return out


def newton_check(x, y, m, kappa_s, gamma, msteps, z, row0=0):
    """Per point of the rows x n_r array z (row r at phi_j, j = row0 + r): the FP64 Newton
    correction |F/F'| (Sec. 3.2; to first order the distance to the zero of F) and the lens
    map w (Sec. 3.1).  Disc field.  Returns (step [rows, n_r] float64, w like z)."""
    x, y, m = _stars(x, y, m)
    zz = np.ascontiguousarray(z, dtype=np.complex128)
    if zz.ndim != 2:
        raise ValueError("z must be rows x n_r")
    rows, nr = zz.shape
    step = np.zeros((rows, nr), dtype=np.float64)
    w = np.zeros_like(zz)
    _load().orc_newton_check(_d(x), _d(y), _d(m), len(x), float(kappa_s), float(gamma), int(msteps), int(row0),
                             rows, nr, zz.view(np.float64).ctypes.data_as(_DP), _d(step),
                             w.view(np.float64).ctypes.data_as(_DP))
    return step, w


def feature_mask(ncc):
    a = np.ascontiguousarray(ncc, dtype=np.int32)
    H, W = a.shape
    out = np.zeros((H, W), dtype=np.uint8)
    _load().orc_feature_mask(a.ctypes.data_as(_I32P), W, H, out.ctypes.data_as(_U8P))
    return out


def distance_map(ncc, pixel, method="separable"):
    """Distance from each pixel to the nearest caustic pixel (Sec. 5.2), FP64 [H, W]."""
    a = np.ascontiguousarray(ncc, dtype=np.int32)
    H, W = a.shape
    out = np.zeros((H, W), dtype=np.float64)
    fn = _load().orc_distance_map_brute if method == "brute" else _load().orc_distance_map_separable
    fn(a.ctypes.data_as(_I32P), W, H, float(pixel), out.ctypes.data_as(_DP))
    return out


def moving_distance_map(ncc, pixel, angle):
    """Distance along direction angle (radians from +x) to the first caustic pixel (Sec. 5.2);
    +inf when the ray leaves the map first.  FP64 [H, W]."""
    a = np.ascontiguousarray(ncc, dtype=np.int32)
    H, W = a.shape
    out = np.zeros((H, W), dtype=np.float64)
    _load().orc_moving_distance_map(a.ctypes.data_as(_I32P), W, H, float(pixel), float(angle),
                                    out.ctypes.data_as(_DP))
    return out
