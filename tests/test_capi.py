"""Host-side checks of the C ABI (no GPU needed): the library builds and loads, and it
exports every function that include/cc.h declares; the binding declares the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_02121_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_five_calls():
    names = _declared()
    for n in ["cc_field_create", "cc_critical_curves", "cc_map_caustics", "cc_crossing_map", "cc_distance_map"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_header(lib):
    from paper_2506_02121_gb300 import cc
    assert sorted(cc.EXPORTED) == _declared()


def test_host_only_calls(lib):
    from paper_2506_02121_gb300 import cc
    o = cc.cc_options_default()
    assert o.tol_abs == 1e-9 and o.precision == cc.CC_MIXED
    assert cc.cc_version().startswith("ccgpu")
    # banded maps: 64-row feature words, chunk summaries and neighbours (8 B each per chunk and
    # column) and a 2^16-entry square-root table; wider maps keep two int32 planes
    assert cc.cc_distance_map_workspace_bytes(4096, 4096) >= 64 * 4096 * 24 + 65536 * 8
    assert cc.cc_distance_map_workspace_bytes(4096, 4096) < 4096 * 4096
    assert cc.cc_distance_map_workspace_bytes(33000, 3) >= 2 * 33000 * 3 * 4
    with pytest.raises(cc.CCError) as e:
        cc.cc_distance_map_workspace_bytes(0, 5)
    assert e.value.status == cc.CC_EINVAL


def test_degenerate_field_rejected_before_any_device_work(lib):
    import numpy as np
    from paper_2506_02121_gb300 import cc
    with pytest.raises(cc.CCError) as e:
        cc.cc_field_create(np.zeros(1), np.zeros(1), np.ones(1), 0.2, 0.8)
    assert e.value.status == cc.CC_EDEGENERATE
    with pytest.raises(cc.CCError) as e:
        cc.cc_field_create(np.zeros(1), np.zeros(1), -np.ones(1), 0.0, 0.3)
    assert e.value.status == cc.CC_EINVAL


def test_rect_options_rejected_before_any_device_work(lib):
    import numpy as np
    from paper_2506_02121_gb300 import cc
    x, y, m = np.zeros(1), np.zeros(1), np.ones(1)
    for kw, status in [(dict(kappa_star=0.0, c1=2.0, c2=1.0), cc.CC_EINVAL),
                       (dict(kappa_star=0.3, c1=-2.0, c2=1.0), cc.CC_EINVAL),
                       (dict(kappa_star=0.3, c1=2.0, c2=1.0, t=8), cc.CC_EINVAL),
                       (dict(kappa_star=0.3, c1=2.0, c2=1.0, t=cc.CC_RECT_MAX_T + 2), cc.CC_EINVAL),
                       # a square with t - 1 = 8: (t - 1) pi/4 is a multiple of pi
                       (dict(kappa_star=0.3, c1=2.0, c2=2.0, t=9), cc.CC_EDEGENERATE)]:
        o = cc.rect_options(**kw)
        with pytest.raises(cc.CCError) as e:
            cc.cc_field_create(x, y, m, 0.0, 0.3, o)
        assert e.value.status == status, kw
    o = cc.cc_options_default()
    o.field_shape = 7
    with pytest.raises(cc.CCError) as e:
        cc.cc_field_create(x, y, m, 0.0, 0.3, o)
    assert e.value.status == cc.CC_EINVAL


def test_root_refresh_default_and_range(lib):
    import numpy as np
    from paper_2506_02121_gb300 import cc
    o = cc.cc_options_default()
    assert o.root_refresh == 64 and o.row_ctas == 0
    x, y, m = np.zeros(1), np.zeros(1), np.ones(1)
    for bad in (-1, 4097):
        o = cc.cc_options_default()
        o.root_refresh = bad
        with pytest.raises(cc.CCError) as e:
            cc.cc_field_create(x, y, m, 0.0, 0.3, o)
        assert e.value.status == cc.CC_EINVAL, bad
