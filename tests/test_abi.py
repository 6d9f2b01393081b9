"""CPU checks of the boundary: libtfx.so builds for sm_103a, loads, exports
every function include/tfx.h declares, and rejects bad arguments before any
launch (these calls never reach the GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_08624_gb300 import build, _native
    build.build()
    return _native.lib()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "tfx.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tfx_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    from paper_2504_08624_gb300 import _native
    names = declared_functions()
    assert len(names) >= 10
    assert set(names) == set(_native.EXPORTS)
    for n in names:
        assert hasattr(lib, n), f"libtfx.so does not export {n}"


def test_strerror_and_version(lib):
    assert lib.tfx_strerror(0) == b"TFX_OK"
    for code in range(-7, 0):
        assert lib.tfx_strerror(code).startswith(b"TFX_ERR_")
    assert lib.tfx_version() == 0x000100


def test_argument_errors_need_no_gpu(lib):
    from paper_2504_08624_gb300 import _native as N
    good = N.StageList([("sos", [[1, 0, 0, 1, -0.5, 0.1]])])
    p = ctypes.c_void_p()
    # negative sizes, bad ld
    assert lib.tfx_plan_create(ctypes.byref(p), -1, 10, 10, good.arr, 1, 0) == -1
    assert lib.tfx_plan_create(ctypes.byref(p), 1, 10, 5, good.arr, 1, 0) == -1
    # a0 == 0 -> invalid; unstable pole -> TFX_ERR_UNSTABLE
    bad = N.StageList([("sos", [[1, 0, 0, 0, 0, 0]])])
    assert lib.tfx_plan_create(ctypes.byref(p), 1, 10, 10, bad.arr, 1, 0) == -1
    uns = N.StageList([("sos", [[1, 0, 0, 1, -2.0, 1.0]])])   # double pole at z = 1
    assert lib.tfx_plan_create(ctypes.byref(p), 1, 10, 10, uns.arr, 1, 0) == -2
    uns2 = N.StageList([("sos", [[1, 0, 0, 1, 0.0, 1.01]])])  # |p| > 1
    assert lib.tfx_plan_create(ctypes.byref(p), 1, 10, 10, uns2.arr, 1, 0) == -2
    nan = N.StageList([("fir", [1.0, float("nan")])])
    assert lib.tfx_plan_create(ctypes.byref(p), 1, 10, 10, nan.arr, 1, 0) == -1
    # unknown flag bits
    assert lib.tfx_plan_create(ctypes.byref(p), 1, 10, 10, good.arr, 1, 1 << 20) == -1
    # workspace size query for invalid input
    assert lib.tfx_chain_workspace_size(1, 10, 5, good.arr, 1) == ctypes.c_size_t(-1).value
    # empty problems are a no-op before any device work
    assert lib.tfx_chain(None, None, 0, 100, 100, good.arr, 1, None, 0, None) == 0
    assert lib.tfx_chain(None, None, 4, 0, 1, good.arr, 1, None, 0, None) == 0
    # null buffers for a non-empty problem
    assert lib.tfx_chain(None, None, 4, 10, 10, good.arr, 1, None, 0, None) == -1
    # partially overlapping x / y
    buf = (ctypes.c_float * 64)()
    base = ctypes.addressof(buf)
    assert lib.tfx_chain(ctypes.c_void_p(base), ctypes.c_void_p(base + 8), 1, 10, 10, good.arr, 1,
                         None, 0, None) == -1


def test_header_constants_match_binding():
    from paper_2504_08624_gb300 import _native as N
    txt = open(os.path.join(ROOT, "include", "tfx.h")).read()
    for name, val in [("TFX_PLAN_FIR_CUDA_CORES", N.TFX_PLAN_FIR_CUDA_CORES),
                      ("TFX_PLAN_UNFUSED", N.TFX_PLAN_UNFUSED),
                      ("TFX_PLAN_FIR_BF16_PLAIN", N.TFX_PLAN_FIR_BF16_PLAIN),
                      ("TFX_PLAN_FIR_BF16_SPLIT", N.TFX_PLAN_FIR_BF16_SPLIT),
                      ("TFX_PLAN_SCAN_WARP_TILES", N.TFX_PLAN_SCAN_WARP_TILES),
                      ("TFX_PLAN_TEST_DROP_PUBLISH", N.TFX_PLAN_TEST_DROP_PUBLISH)]:
        m = re.search(rf"#define {name} (\d+)u", txt)
        assert m and int(m.group(1)) == val
    for code, name in N.STATUS.items():
        assert re.search(rf"{name} = {code}\b", txt), name
