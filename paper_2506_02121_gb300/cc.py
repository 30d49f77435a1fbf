"""ctypes binding of libccgpu (include/cc.h): the same calls, argument marshalling only.

Every function takes PyTorch CUDA tensors for device buffers (torch is used for device
memory and streams only) and forwards raw pointers to the C ABI; every step of the
computation runs in the CUDA kernels of the library.  There is no CPU fallback: if the
library is missing or cannot be loaded, importing this module raises.

Layouts follow include/cc.h: complex arrays are torch.complex128 (interleaved re, im
doubles), the chain matrix is [(m+1), n_r] with row j at phi_j = 2 pi j / m, maps are
[H, W] with row 0 at y0.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccgpu.so")

CC_OK, CC_EINVAL, CC_ENOMEM, CC_ENOCONV, CC_EDEGENERATE, CC_ECUDA = range(6)
CC_MIXED, CC_FP64 = 0, 1
CC_HP_DFLOAT, CC_HP_FP64 = 0, 1
CC_FIELD_DISC, CC_FIELD_RECT = 0, 1
CC_RECT_MAX_T = 129
_NAMES = {0: "CC_OK", 1: "CC_EINVAL", 2: "CC_ENOMEM", 3: "CC_ENOCONV", 4: "CC_EDEGENERATE", 5: "CC_ECUDA"}


class CCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_NAMES.get(status, status)}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("tol_abs", ctypes.c_double), ("mu_max", ctypes.c_double), ("tol_cert", ctypes.c_double),
                ("max_iter_cold", ctypes.c_int32), ("max_iter_warm", ctypes.c_int32),
                ("max_polish", ctypes.c_int32), ("precision", ctypes.c_int32), ("hp_arith", ctypes.c_int32),
                ("subchains", ctypes.c_int32), ("predictor", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("far_field", ctypes.c_int32), ("field_shape", ctypes.c_int32), ("rect_t", ctypes.c_int32),
                ("kappa_star", ctypes.c_double), ("rect_c1", ctypes.c_double), ("rect_c2", ctypes.c_double),
                ("rect_eps", ctypes.c_double), ("rect_s", ctypes.c_double), ("row_ctas", ctypes.c_int32),
                ("root_refresh", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("n_roots", ctypes.c_int64), ("subchains", ctypes.c_int64),
                ("root_iterations", ctypes.c_int64), ("cold_root_iterations", ctypes.c_int64),
                ("unconverged", ctypes.c_int64), ("polish_passes", ctypes.c_int64),
                ("uncertified", ctypes.c_int64), ("seam_ambiguous", ctypes.c_int64),
                ("max_iter_row", ctypes.c_int32), ("max_err_est", ctypes.c_double),
                ("trace_ms", ctypes.c_float), ("join_ms", ctypes.c_float), ("polish_ms", ctypes.c_float),
                ("rescued_points", ctypes.c_int64), ("jumped", ctypes.c_int64),
                ("star_terms", ctypes.c_int64), ("far_evals", ctypes.c_int64),
                ("root_terms", ctypes.c_int64), ("split_redone_rows", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2506_02121_gb300.build.build()")
_lib = ctypes.CDLL(LIB_PATH)

_vp, _i64, _i32, _dbl, _sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
_sig = {
    "cc_options_default": ([ctypes.POINTER(Options)], ctypes.c_int),
    "cc_field_create": ([_vp, _vp, _vp, _i64, _dbl, _dbl, ctypes.POINTER(Options), ctypes.POINTER(_vp)], ctypes.c_int),
    "cc_field_destroy": ([_vp], ctypes.c_int),
    "cc_field_size": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], ctypes.c_int),
    "cc_critical_curves_workspace_bytes": ([_vp, _i64, ctypes.POINTER(_sz)], ctypes.c_int),
    "cc_critical_curves": ([_vp, _i64, _vp, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "cc_field_report": ([_vp, ctypes.POINTER(Report)], ctypes.c_int),
    "cc_map_caustics": ([_vp, _vp, _i64, _vp, _vp], ctypes.c_int),
    "cc_crossing_map": ([_vp, _i64, _i64, _dbl, _dbl, _dbl, _dbl, _i32, _i32, _vp, _vp], ctypes.c_int),
    "cc_distance_map_workspace_bytes": ([_i32, _i32, ctypes.POINTER(_sz)], ctypes.c_int),
    "cc_distance_map": ([_vp, _i32, _i32, _dbl, _vp, _vp, _sz, _vp], ctypes.c_int),
    "cc_distance_map_static": ([_vp, _i32, _i32, _dbl, _vp, _vp], ctypes.c_int),
    "cc_moving_distance_map": ([_vp, _i32, _i32, _dbl, _dbl, _vp, _vp], ctypes.c_int),
    "cc_batch_create": ([ctypes.POINTER(_vp), _i32, ctypes.POINTER(_i64), _i32, _i32, ctypes.POINTER(_vp)], ctypes.c_int),
    "cc_batch_workspace_bytes": ([_vp, ctypes.POINTER(_sz)], ctypes.c_int),
    "cc_batch_bind": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _sz], ctypes.c_int),
    "cc_batch_launch": ([_vp, _i32, _vp], ctypes.c_int),
    "cc_batch_report": ([_vp, ctypes.POINTER(Report), ctypes.POINTER(Report)], ctypes.c_int),
    "cc_batch_info": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)], ctypes.c_int),
    "cc_batch_destroy": ([_vp], ctypes.c_int),
    "cc_last_error": ([], ctypes.c_char_p),
    "cc_version": ([], ctypes.c_char_p),
}
for _name, (_args, _res) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res

EXPORTED = tuple(_sig)


def _check(status: int, allow=()):
    if status != CC_OK and status not in allow:
        raise CCError(status, _lib.cc_last_error().decode())
    return status


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _dev_ptr(t, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return _ptr(t)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def cc_version() -> str:
    return _lib.cc_version().decode()


def cc_options_default() -> Options:
    o = Options()
    _check(_lib.cc_options_default(ctypes.byref(o)))
    return o


def rect_options(kappa_star: float, c1: float, c2: float, t: int = 0, base: Options | None = None) -> Options:
    """Options for a rectangular microlens field |Re z| <= c1, |Im z| <= c2 (Sec. 4.2) whose
    smooth sheet has convergence kappa_star; t = 0 picks the truncation order by the
    Appendix B rule."""
    o = cc_options_default() if base is None else base
    o.field_shape = CC_FIELD_RECT
    o.kappa_star = float(kappa_star)
    o.rect_c1 = float(c1)
    o.rect_c2 = float(c2)
    o.rect_t = int(t)
    return o


class Field:
    """Owner of a cc_field handle (stars resident on the device)."""

    def __init__(self, handle, n, n_roots):
        self._h = handle
        self.n = n
        self.n_roots = n_roots  # 2N (disc) or 2N + t - 1 (rectangular field)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("field was destroyed")
        return self._h

    def __del__(self):
        try:
            cc_field_destroy(self)
        except Exception:
            pass


def cc_field_create(x, y, mass, kappa_s: float, gamma: float, opt: Options | None = None) -> Field:
    """x, y, mass: float64 tensors (CPU or CUDA) or numpy arrays of length N."""
    import numpy as np

    def as_t(a):
        if isinstance(a, torch.Tensor):
            return a.detach().to(torch.float64).contiguous()
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))

    tx, ty, tm = as_t(x), as_t(y), as_t(mass)
    n = int(tx.numel())
    if ty.numel() != n or tm.numel() != n:
        raise ValueError("x, y, mass must have equal length")
    h = ctypes.c_void_p()
    _check(_lib.cc_field_create(_ptr(tx), _ptr(ty), _ptr(tm), n, float(kappa_s), float(gamma),
                                ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    ns, nr = _i64(), _i64()
    _check(_lib.cc_field_size(h, ctypes.byref(ns), ctypes.byref(nr)))
    return Field(h, n, nr.value)


def cc_field_destroy(field: Field):
    if field._h is not None:
        _lib.cc_field_destroy(field._h)
        field._h = None


def cc_field_size(field: Field):
    ns, nr = _i64(), _i64()
    _check(_lib.cc_field_size(field.handle, ctypes.byref(ns), ctypes.byref(nr)))
    return ns.value, nr.value


def cc_critical_curves_workspace_bytes(field: Field, m: int) -> int:
    b = _sz()
    _check(_lib.cc_critical_curves_workspace_bytes(field.handle, int(m), ctypes.byref(b)))
    return b.value


def cc_critical_curves(field: Field, m: int, z_out, w_out=None, iters_out=None, workspace=None, stream=None):
    rows = int(m) + 1
    shape = (rows, field.n_roots)
    zp = _dev_ptr(z_out, torch.complex128, shape)
    wp = _dev_ptr(w_out, torch.complex128, shape) if w_out is not None else None
    ip = _dev_ptr(iters_out, torch.int32, shape) if iters_out is not None else None
    if workspace is None:
        raise ValueError("workspace tensor required (see cc_critical_curves_workspace_bytes)")
    _check(_lib.cc_critical_curves(field.handle, int(m), zp, wp, ip, _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), _stream(stream)))


def cc_field_report(field: Field):
    """Returns (status, report dict); status is CC_OK or CC_ENOCONV."""
    r = Report()
    st = _check(_lib.cc_field_report(field.handle, ctypes.byref(r)), allow=(CC_ENOCONV,))
    return st, r.as_dict()


def cc_map_caustics(field: Field, z, w_out, stream=None):
    zp = _dev_ptr(z, torch.complex128)
    wp = _dev_ptr(w_out, torch.complex128, tuple(z.shape))
    _check(_lib.cc_map_caustics(field.handle, zp, z.numel(), wp, _stream(stream)))


def cc_crossing_map(w, x0: float, x1: float, y0: float, y1: float, W: int, H: int, ncc_out, stream=None):
    """w: [rows, n_r] complex128 caustic vertices; ncc_out: [H, W] int32."""
    if w.dim() != 2:
        raise ValueError("w must be [rows, n_r]")
    wp = _dev_ptr(w, torch.complex128)
    np_ = _dev_ptr(ncc_out, torch.int32, (H, W))
    _check(_lib.cc_crossing_map(wp, w.shape[0], w.shape[1], float(x0), float(x1), float(y0), float(y1),
                                int(W), int(H), np_, _stream(stream)))


def cc_distance_map_workspace_bytes(W: int, H: int) -> int:
    b = _sz()
    _check(_lib.cc_distance_map_workspace_bytes(int(W), int(H), ctypes.byref(b)))
    return b.value


def cc_distance_map(ncc, pixel: float, d_out, workspace, stream=None):
    H, W = ncc.shape
    _check(_lib.cc_distance_map(_dev_ptr(ncc, torch.int32), int(W), int(H), float(pixel),
                                _dev_ptr(d_out, torch.float64, (H, W)), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)))


def cc_moving_distance_map(ncc, pixel: float, angle: float, d_out, stream=None):
    """Distance along direction angle (radians from +x) to the first caustic pixel; +inf
    when the ray leaves the map first (Sec. 5.2)."""
    H, W = ncc.shape
    _check(_lib.cc_moving_distance_map(_dev_ptr(ncc, torch.int32), int(W), int(H), float(pixel), float(angle),
                                       _dev_ptr(d_out, torch.float64, (H, W)), _stream(stream)))


def moving_distance_map(ncc, pixel, angle, stream=None):
    H, W = ncc.shape
    out = torch.empty((H, W), dtype=torch.float64, device="cuda")
    cc_moving_distance_map(ncc, pixel, angle, out, stream)
    return out


DISTANCE_MAP_STATIC_MAX_PIXELS = 1048576


def cc_distance_map_static(ncc, pixel: float, d_out, stream=None):
    """Distance map for callers that cannot allocate device memory: the library's fixed
    static scratch replaces the workspace (maps up to DISTANCE_MAP_STATIC_MAX_PIXELS
    pixels).  Allocates nothing; ncc and d_out are the caller's buffers."""
    H, W = ncc.shape
    _check(_lib.cc_distance_map_static(_dev_ptr(ncc, torch.int32), int(W), int(H), float(pixel),
                                       _dev_ptr(d_out, torch.float64, (H, W)), _stream(stream)))


class Batch:
    """Owner of a cc_batch handle; keeps its fields, outputs and workspace alive."""

    def __init__(self, handle, fields, msteps):
        self._h = handle
        self.fields = list(fields)
        self.msteps = list(msteps)
        self.z = self.w = self.workspace = None

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("batch was destroyed")
        return self._h

    def __del__(self):
        try:
            cc_batch_destroy(self)
        except Exception:
            pass


def cc_batch_create(fields, msteps, block_threads: int = 0, items_per_cta: int = 0) -> Batch:
    n = len(fields)
    hs = (ctypes.c_void_p * n)(*[f.handle for f in fields])
    ms = (ctypes.c_int64 * n)(*[int(v) for v in msteps])
    h = ctypes.c_void_p()
    _check(_lib.cc_batch_create(hs, n, ms, int(block_threads), int(items_per_cta), ctypes.byref(h)))
    return Batch(h, fields, msteps)


def cc_batch_workspace_bytes(batch: Batch) -> int:
    b = _sz()
    _check(_lib.cc_batch_workspace_bytes(batch.handle, ctypes.byref(b)))
    return b.value


def cc_batch_bind(batch: Batch, z_out, w_out, workspace):
    n = len(batch.fields)
    for f, (fld, m) in enumerate(zip(batch.fields, batch.msteps)):
        _dev_ptr(z_out[f], torch.complex128, (m + 1, fld.n_roots))
        if w_out is not None and w_out[f] is not None:
            _dev_ptr(w_out[f], torch.complex128, (m + 1, fld.n_roots))
    zp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in z_out])
    wp = None
    if w_out is not None:
        wp = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in w_out])
    _check(_lib.cc_batch_bind(batch.handle, zp, wp, _ptr(workspace), workspace.numel() * workspace.element_size()))
    batch.z, batch.w, batch.workspace = z_out, w_out, workspace


def cc_batch_launch(batch: Batch, use_graph: bool = False, stream=None):
    _check(_lib.cc_batch_launch(batch.handle, 1 if use_graph else 0, _stream(stream)))


def cc_batch_report(batch: Batch):
    n = len(batch.fields)
    per = (Report * n)()
    tot = Report()
    st = _check(_lib.cc_batch_report(batch.handle, per, ctypes.byref(tot)), allow=(CC_ENOCONV,))
    return st, [p.as_dict() for p in per], tot.as_dict()


def cc_batch_info(batch: Batch):
    a, b, c = _i32(), _i32(), _i32()
    _check(_lib.cc_batch_info(batch.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"items": a.value, "grid": b.value, "threads": c.value}


def cc_batch_destroy(batch: Batch):
    if batch._h is not None:
        _lib.cc_batch_destroy(batch._h)
        batch._h = None


def batch_critical_curves(fields, msteps, caustics: bool = True, use_graph: bool = False, stream=None,
                          block_threads: int = 0, items_per_cta: int = 0):
    """Plan, bind and launch a batch; returns the Batch (outputs in batch.z / batch.w)."""
    b = cc_batch_create(fields, msteps, block_threads, items_per_cta)
    z = [torch.empty((m + 1, f.n_roots), dtype=torch.complex128, device="cuda") for f, m in zip(fields, msteps)]
    w = [torch.empty_like(t) for t in z] if caustics else None
    ws = workspace(cc_batch_workspace_bytes(b))
    cc_batch_bind(b, z, w, ws)
    cc_batch_launch(b, use_graph, stream)
    return b


# --------------------------------------------------------------------------------------
# Convenience wrappers: allocate outputs and workspaces with torch, then call the ABI.
# --------------------------------------------------------------------------------------

def workspace(nbytes: int, device=None) -> torch.Tensor:
    """A 256-byte-aligned uint8 device buffer (the caching allocator aligns to 512 B)."""
    t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device or "cuda")
    assert t.data_ptr() % 256 == 0
    return t


def critical_curves(field: Field, m: int, caustics: bool = True, iters: bool = False, stream=None):
    """Returns (z, w or None, iters or None) as CUDA tensors; the solve is enqueued on the
    stream and not waited for."""
    rows = int(m) + 1
    z = torch.empty((rows, field.n_roots), dtype=torch.complex128, device="cuda")
    w = torch.empty_like(z) if caustics else None
    it = torch.empty((rows, field.n_roots), dtype=torch.int32, device="cuda") if iters else None
    ws = workspace(cc_critical_curves_workspace_bytes(field, m))
    cc_critical_curves(field, m, z, w, it, ws, stream)
    return z, w, it


def crossing_map(w, x0, x1, y0, y1, W, H, stream=None):
    out = torch.empty((H, W), dtype=torch.int32, device="cuda")
    cc_crossing_map(w, x0, x1, y0, y1, W, H, out, stream)
    return out


def distance_map(ncc, pixel, stream=None):
    H, W = ncc.shape
    out = torch.empty((H, W), dtype=torch.float64, device="cuda")
    ws = workspace(cc_distance_map_workspace_bytes(W, H))
    cc_distance_map(ncc, pixel, out, ws, stream)
    return out
