"""ctypes binding of libtfx.so (declared in include/tfx.h).

Argument marshalling only: every step of the filter path runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libtfx.so")

TFX_STAGE_FIR = 0
TFX_STAGE_SOS = 1

TFX_PLAN_DEFAULT = 0
TFX_PLAN_FIR_CUDA_CORES = 1
TFX_PLAN_UNFUSED = 2
TFX_PLAN_FIR_BF16_PLAIN = 4
TFX_PLAN_FIR_BF16_SPLIT = 8
TFX_PLAN_SCAN_WARP_TILES = 16
TFX_PLAN_TRAINABLE = 32
TFX_PLAN_FIR_FFT = 64
TFX_PLAN_FIR_TC = 128


def TFX_PLAN_FIR_FFT_LOG(m: int) -> int:
    """Plan flag bits fixing the overlap-save transform size at 2^m points (m = 10..14; 14: single-block only)."""
    return (int(m) & 15) << 16


TFX_PLAN_TEST_DROP_PUBLISH = 256
TFX_PLAN_SCAN_LOOKBACK = 512
TFX_PLAN_NO_COMPOSE = 1024

STATUS = {
    0: "TFX_OK", -1: "TFX_ERR_INVALID", -2: "TFX_ERR_UNSTABLE", -3: "TFX_ERR_WORKSPACE",
    -4: "TFX_ERR_CUDA", -5: "TFX_ERR_TIMEOUT", -6: "TFX_ERR_UNSUPPORTED", -7: "TFX_ERR_NOMEM",
    -8: "TFX_ERR_DECAY",
}

# every symbol include/tfx.h declares
EXPORTS = [
    "tfx_plan_create", "tfx_plan_workspace_size", "tfx_plan_launch_count", "tfx_plan_describe", "tfx_plan_execute",
    "tfx_plan_execute_plain",
    "tfx_plan_get_error", "tfx_plan_destroy", "tfx_fir", "tfx_sos", "tfx_chain",
    "tfx_chain_workspace_size", "tfx_cache_clear", "tfx_sos_noalloc", "tfx_strerror", "tfx_version",
    "tfx_chain_host", "tfx_host_cache_clear", "tfx_host_cache_info",
    "tfx_plan_saved_size", "tfx_plan_backward_workspace_size", "tfx_plan_coef_count", "tfx_plan_forward_train",
    "tfx_plan_forward_train_mse", "tfx_plan_forward_train_mse_launch_count",
    "tfx_plan_train_step_mse", "tfx_plan_train_step_mse_launch_count",
    "tfx_plan_backward", "tfx_plan_backward_launch_count", "tfx_mse",
    "tfx_batch_create", "tfx_batch_total_samples", "tfx_batch_clip_offset", "tfx_batch_workspace_size",
    "tfx_batch_launch_count", "tfx_batch_execute", "tfx_batch_get_error", "tfx_batch_destroy",
    "tfx_batch_group_count", "tfx_batch_group_info", "tfx_batch_execute_group", "tfx_batch_clip_info",
    "tfx_design_sections", "tfx_design_device", "tfx_plan_update_sos", "tfx_plan_sos_rows",
    "tfx_fma_probe", "tfx_fma_probe_flops", "tfx_plan_update_coefs", "tfx_plan_update_coefs_launch_count",
]


class TfxError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} ({strerror(code)})" if what else STATUS.get(code, str(code)))


class Stage(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("coef", ctypes.POINTER(ctypes.c_double))]


class Clip(ctypes.Structure):
    _fields_ = [("C", ctypes.c_int64), ("N", ctypes.c_int64), ("st", ctypes.POINTER(Stage)), ("nst", ctypes.c_int32)]


class Design(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("order", ctypes.c_int32), ("f1", ctypes.c_double), ("f2", ctypes.c_double),
                ("fs", ctypes.c_double), ("p1", ctypes.c_double), ("p2", ctypes.c_double),
                ("b", ctypes.c_double * 3)]


DESIGN_KINDS = {"butter_low": 0, "butter_high": 1, "cheby1_low": 2, "peaking": 3, "low_shelf": 4,
                "high_shelf": 5, "biquad_polar": 6}


class BatchParams(ctypes.Structure):
    _fields_ = [("plan_flags", ctypes.c_uint32), ("fir_nb", ctypes.c_int32), ("tc_min_taps", ctypes.c_int32),
                ("fft_m", ctypes.c_int32 * 16)]


_lib = None


def lib():
    """The loaded libtfx (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtfx.so not found at {LIB_PATH}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    i64, i32, u32, vp, sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_size_t
    fp = ctypes.c_void_p
    sp = ctypes.POINTER(Stage)
    L.tfx_plan_create.argtypes = [ctypes.POINTER(vp), i64, i64, i64, sp, i32, u32]
    L.tfx_plan_create.restype = ctypes.c_int
    L.tfx_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    L.tfx_plan_describe.restype = ctypes.c_int
    L.tfx_plan_workspace_size.argtypes = [vp]
    L.tfx_plan_workspace_size.restype = sz
    L.tfx_plan_launch_count.argtypes = [vp]
    L.tfx_plan_launch_count.restype = ctypes.c_int
    L.tfx_plan_execute.argtypes = [vp, fp, fp, vp, sz, vp]
    L.tfx_plan_execute.restype = ctypes.c_int
    L.tfx_plan_execute_plain.argtypes = [vp, fp, fp, vp, sz, vp]
    L.tfx_plan_execute_plain.restype = ctypes.c_int
    L.tfx_plan_get_error.argtypes = [vp]
    L.tfx_plan_get_error.restype = ctypes.c_int
    L.tfx_plan_destroy.argtypes = [vp]
    L.tfx_plan_destroy.restype = None
    dp = ctypes.POINTER(ctypes.c_double)
    L.tfx_fir.argtypes = [fp, fp, i64, i64, i64, dp, i32, vp]
    L.tfx_fir.restype = ctypes.c_int
    L.tfx_sos.argtypes = [fp, fp, i64, i64, i64, dp, i32, vp]
    L.tfx_sos.restype = ctypes.c_int
    L.tfx_chain.argtypes = [fp, fp, i64, i64, i64, sp, i32, vp, sz, vp]
    L.tfx_chain.restype = ctypes.c_int
    L.tfx_chain_host.argtypes = [fp, fp, i64, i64, i64, sp, i32, vp]
    L.tfx_chain_host.restype = ctypes.c_int
    L.tfx_host_cache_clear.argtypes = []
    L.tfx_host_cache_clear.restype = None
    L.tfx_host_cache_info.argtypes = [ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.tfx_host_cache_info.restype = ctypes.c_int
    L.tfx_chain_workspace_size.argtypes = [i64, i64, i64, sp, i32]
    L.tfx_chain_workspace_size.restype = sz
    L.tfx_sos_noalloc.argtypes = [fp, fp, i64, i64, i64, dp, i32, vp]
    L.tfx_sos_noalloc.restype = ctypes.c_int
    L.tfx_cache_clear.argtypes = []
    L.tfx_cache_clear.restype = None
    L.tfx_plan_saved_size.argtypes = [vp]
    L.tfx_plan_saved_size.restype = sz
    L.tfx_plan_backward_workspace_size.argtypes = [vp]
    L.tfx_plan_backward_workspace_size.restype = sz
    L.tfx_plan_coef_count.argtypes = [vp]
    L.tfx_plan_coef_count.restype = i64
    L.tfx_plan_forward_train.argtypes = [vp, fp, fp, vp, sz, vp, sz, vp]
    L.tfx_plan_forward_train.restype = ctypes.c_int
    L.tfx_plan_forward_train_mse.argtypes = [vp, fp, fp, fp, fp, ctypes.POINTER(ctypes.c_double), vp, sz, vp, sz, vp]
    L.tfx_plan_forward_train_mse.restype = ctypes.c_int
    L.tfx_plan_forward_train_mse_launch_count.argtypes = [vp]
    L.tfx_plan_forward_train_mse_launch_count.restype = ctypes.c_int
    L.tfx_plan_train_step_mse.argtypes = [vp, fp, fp, fp, fp, ctypes.POINTER(ctypes.c_double), fp,
                                          ctypes.POINTER(ctypes.c_double), vp, sz, vp, sz, vp]
    L.tfx_plan_train_step_mse.restype = ctypes.c_int
    L.tfx_plan_train_step_mse_launch_count.argtypes = [vp, i32, i32]
    L.tfx_plan_train_step_mse_launch_count.restype = ctypes.c_int
    L.tfx_plan_backward.argtypes = [vp, fp, fp, fp, fp, vp, sz, vp, sz, vp]
    L.tfx_plan_backward.restype = ctypes.c_int
    L.tfx_plan_backward_launch_count.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.tfx_plan_backward_launch_count.restype = ctypes.c_int
    L.tfx_mse.argtypes = [fp, fp, fp, i64, i64, i64, fp, vp]
    L.tfx_mse.restype = ctypes.c_int
    L.tfx_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Clip), i32, ctypes.POINTER(BatchParams)]
    L.tfx_batch_create.restype = ctypes.c_int
    L.tfx_batch_total_samples.argtypes = [vp]
    L.tfx_batch_total_samples.restype = i64
    L.tfx_batch_clip_offset.argtypes = [vp, i32]
    L.tfx_batch_clip_offset.restype = i64
    L.tfx_batch_workspace_size.argtypes = [vp]
    L.tfx_batch_workspace_size.restype = sz
    L.tfx_batch_launch_count.argtypes = [vp]
    L.tfx_batch_launch_count.restype = ctypes.c_int
    L.tfx_batch_execute.argtypes = [vp, fp, fp, vp, sz, vp]
    L.tfx_batch_execute.restype = ctypes.c_int
    L.tfx_batch_get_error.argtypes = [vp]
    L.tfx_batch_get_error.restype = ctypes.c_int
    L.tfx_batch_destroy.argtypes = [vp]
    L.tfx_batch_destroy.restype = None
    L.tfx_batch_clip_info.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.tfx_batch_clip_info.restype = ctypes.c_int
    L.tfx_batch_group_count.argtypes = [vp]
    L.tfx_batch_group_count.restype = ctypes.c_int
    ip32, ip64 = ctypes.POINTER(i32), ctypes.POINTER(i64)
    L.tfx_batch_group_info.argtypes = [vp, i32, ip32, ip32, ip64, ip64, ctypes.POINTER(ctypes.c_double)]
    L.tfx_batch_group_info.restype = ctypes.c_int
    L.tfx_batch_execute_group.argtypes = [vp, i32, fp, fp, vp, sz, vp]
    L.tfx_batch_execute_group.restype = ctypes.c_int
    L.tfx_design_sections.argtypes = [ctypes.POINTER(Design)]
    L.tfx_design_sections.restype = ctypes.c_int
    L.tfx_design_device.argtypes = [vp, i32, vp, vp, vp, vp]
    L.tfx_design_device.restype = ctypes.c_int
    L.tfx_plan_update_sos.argtypes = [vp, vp, vp]
    L.tfx_plan_update_sos.restype = ctypes.c_int
    L.tfx_plan_update_coefs.argtypes = [vp, vp, vp]
    L.tfx_plan_update_coefs.restype = ctypes.c_int
    L.tfx_plan_update_coefs_launch_count.argtypes = [vp]
    L.tfx_plan_update_coefs_launch_count.restype = ctypes.c_int
    L.tfx_plan_sos_rows.argtypes = [vp]
    L.tfx_plan_sos_rows.restype = i64
    L.tfx_fma_probe.argtypes = [fp, i32, i32, i32, i32, vp]
    L.tfx_fma_probe.restype = ctypes.c_int
    L.tfx_fma_probe_flops.argtypes = [i32, i32, i32, i32]
    L.tfx_fma_probe_flops.restype = ctypes.c_double
    L.tfx_strerror.argtypes = [ctypes.c_int]
    L.tfx_strerror.restype = ctypes.c_char_p
    L.tfx_version.restype = ctypes.c_int
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().tfx_strerror(int(code)).decode()
    except Exception:  # pragma: no cover
        return STATUS.get(code, str(code))


def check(rc: int, what: str) -> None:
    if rc != 0:
        raise TfxError(rc, what)


class StageList:
    """Stage array in the C layout; keeps the FP64 coefficient buffers alive."""

    def __init__(self, stages):
        self._keep = []
        items = []
        for kind, coef in stages:
            if kind == "fir":
                c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).ravel())
                items.append((TFX_STAGE_FIR, c.size, c))
            elif kind == "sos":
                c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1, 6))
                items.append((TFX_STAGE_SOS, c.shape[0], c))
            else:
                raise ValueError(f"unknown stage kind {kind!r} (use 'fir' or 'sos')")
            self._keep.append(c)
        self.n = len(items)
        self.arr = (Stage * max(1, self.n))()
        for i, (k, n, c) in enumerate(items):
            self.arr[i].kind = k
            self.arr[i].n = n
            self.arr[i].coef = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
