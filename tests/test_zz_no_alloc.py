"""The allocation-free distance map, for callers that cannot allocate device memory.

Such callers (a plugin whose host application owns all device memory, a process whose
device-memory budget is fully reserved, a loop that must never enter the allocator)
cannot pass the workspace that cc_distance_map needs; cc_distance_map_static uses the
library's fixed static scratch instead.  This file is collected last so that a run that
stops at the first failure has already run every other test; it also passes on its own
in a fresh process, where its first call does the per-device set-up.
"""
import numpy as np
import pytest
import torch

from paper_2506_02121_gb300 import cc, synth

pytestmark = pytest.mark.gpu


def _ncc_map(seed, H, W):
    u = synth.uniform(seed, H * W).reshape(H, W)
    ncc = (u < 0.002).astype(np.int32)
    ncc[H // 5: H // 2, W // 4: (3 * W) // 4] += 1
    ncc[(2 * H) // 3:, : W // 3] += 3
    return torch.from_numpy(ncc).cuda()


def test_static_scratch_matches_workspace_version_on_consecutive_calls():
    pixel = 20.0 / 1024
    # Two calls in a row on different maps: the second reuses the shared static array
    # with the first call's contents still in it.
    for seed, (H, W) in [(11, (1024, 1024)), (12, (517, 983))]:
        ncc = _ncc_map(seed, H, W)
        ref = cc.distance_map(ncc, pixel)  # caller-provided workspace version
        out = torch.full((H, W), -1.0, dtype=torch.float64, device="cuda")
        cc.cc_distance_map_static(ncc, pixel, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)  # bit-exact, as every distance-map comparison here


def test_static_scratch_call_allocates_no_device_memory():
    H, W = 777, 1301
    ncc = _ncc_map(13, H, W)
    out = torch.empty((H, W), dtype=torch.float64, device="cuda")
    pixel = 20.0 / 1024
    cc.cc_distance_map_static(ncc, pixel, out)  # warm-up: per-context set-up, module load
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    cc.cc_distance_map_static(ncc, pixel, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == reserved0
    assert free1 == free0


def test_static_scratch_rejects_maps_beyond_its_limit():
    H, W = 1025, 1024
    ncc = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    out = torch.empty((H, W), dtype=torch.float64, device="cuda")
    with pytest.raises(cc.CCError) as e:
        cc.cc_distance_map_static(ncc, 0.1, out)
    assert e.value.status == cc.CC_EINVAL
    assert "CC_DISTANCE_MAP_STATIC_MAX_PIXELS" in str(e.value)
