"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/fmm.h (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import paper_2002_04894_gb300 as fmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z0-9_]+)\s*\(", text)) - {"fmm_alloc_fn", "fmm_free_fn"})


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("fmm_plan", "fmm_eval", "fmm_destroy", "fmm_direct", "fmm_strerror"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    lib = fmm.load()
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(fmm.EXPORTS) == set(declared_symbols())


def test_strerror_without_gpu():
    lib = fmm.load()
    assert fmm.fmm_strerror(0) == "success"
    assert "non-finite" in fmm.fmm_strerror(-3)
    assert fmm.fmm_strerror(12345) == "unknown status"


def test_invalid_arguments_rejected_before_any_device_work():
    """Argument checks run on the host: no CUDA call is made for these."""
    lib = fmm.load()
    opts = fmm.fmm_opts(3, 4, 0.5, 0, 0)
    h = ctypes.c_void_p()
    import numpy as np
    pts = np.zeros((4, 3))
    for bad in (fmm.fmm_opts(-1, 4, 0.5, 0, 0), fmm.fmm_opts(25, 4, 0.5, 0, 0),
                fmm.fmm_opts(3, 21, 0.5, 0, 0), fmm.fmm_opts(3, 4, 1.0, 0, 0),
                fmm.fmm_opts(3, 4, -0.1, 0, 0), fmm.fmm_opts(3, 4, float("nan"), 0, 0),
                fmm.fmm_opts(3, 4, 0.5, 7, 0), fmm.fmm_opts(3, 4, 0.5, 0, 64),
                fmm.fmm_opts(3, 4, 0.5, 0, fmm.FMM_FLAG_ETA, 1.5),
                fmm.fmm_opts(3, 4, 0.5, 0, fmm.FMM_FLAG_ETA, -0.25),
                fmm.fmm_opts(3, 4, 0.5, 0, fmm.FMM_FLAG_ETA, float("nan")),
                fmm.fmm_opts(4, 4, 0.5, 0, 0, 1.0, 3), fmm.fmm_opts(4, 4, 0.5, 0, 0, 1.0, 4),
                fmm.fmm_opts(4, 4, 0.5, 0, 0, 1.0, -1)):
        assert lib.fmm_plan(pts.ctypes.data, 4, 0, ctypes.byref(bad), None, None, ctypes.byref(h)) == -1
        assert h.value is None
    assert lib.fmm_plan(pts.ctypes.data, 0, 0, ctypes.byref(opts), None, None, ctypes.byref(h)) == -1
    assert lib.fmm_plan(pts.ctypes.data, 4, 5, ctypes.byref(opts), None, None, ctypes.byref(h)) == -1
    assert lib.fmm_plan(None, 4, 0, ctypes.byref(opts), None, None, ctypes.byref(h)) == -1
    assert lib.fmm_eval(None, None, None, None, None) == -1
    assert lib.fmm_plan_stats(None, None) == -1
    lib.fmm_destroy(None)


def test_launch_counter_starts_at_zero_without_gpu_work():
    assert fmm.fmm_kernel_launches() == 0
