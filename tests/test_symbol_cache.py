"""Host logic of the static-scratch address cache (csrc/symbol_cache.h), on the CPU.

cc_distance_map_static keeps the device address of its static scratch per CUDA context:
an address found in one context must not be reused in a later one (a reset device loads
its module anew).  The header is plain C++, so a small g++ program drives it with a fake
lookup and checks that the key is the context, not the device.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_02121_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "symbol_cache.h"

static int lookups = 0;
static char arena[16];

int main() {
    ccg::SymbolAddressCache<4> c;
    void* p = nullptr;
    auto look = [](void** a) -> int { *a = arena + (lookups++ % 16); return 0; };
    // first call in context 7 looks the address up; later calls in it do not
    if (c.get(7, look, &p) || p != arena + 0 || lookups != 1) return 1;
    if (c.get(7, look, &p) || p != arena + 0 || lookups != 1) return 2;
    // a new context (e.g. after a device reset) looks it up again, and gets its own entry
    if (c.get(8, look, &p) || p != arena + 1 || lookups != 2) return 3;
    if (c.get(7, look, &p) || p != arena + 0 || lookups != 2) return 4;
    // a failed lookup is not cached and passes its error on
    auto fail = [](void** a) -> int { *a = nullptr; return 5; };
    if (c.get(9, fail, &p) != 5 || c.size() != 2) return 5;
    // a full table replaces entries in turn and stays correct for the contexts it holds
    for (unsigned long long k = 10; k < 20; k++) {
        if (c.get(k, look, &p)) return 6;
        void* q = nullptr;
        int before = lookups;
        if (c.get(k, look, &q) || q != p || lookups != before) return 7;
    }
    if (c.size() != 4) return 8;
    std::puts("ok");
    return 0;
}
"""


def test_address_cache_is_keyed_by_context(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "t.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "t"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe), "-pthread"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
