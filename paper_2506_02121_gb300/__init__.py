"""GB300-native microlensing critical curves, caustics and caustic-crossing maps.

The compute path is the CUDA library ``libccgpu.so`` (hand-written kernels for sm_103a)
behind the C ABI declared in ``include/cc.h``; :mod:`paper_2506_02121_gb300.cc` is the
thin ctypes binding with the same names.  Submodules load lazily so that the seeded input
generators (:mod:`paper_2506_02121_gb300.synth`) import without a GPU.
"""
__all__ = ["cc", "synth"]


def __getattr__(name):
    if name in ("cc", "synth"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
