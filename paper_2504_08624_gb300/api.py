"""Python API over libtfx: filter chains on [channels x samples] FP32 tensors.

TorchFX (arXiv 2504.08624, Sec. 3) applies FIR and IIR filters to every
channel of a signal and chains them with a pipe operator; this module exposes
the same operation: ``chain(x, stages)`` with stages applied in list order,
plus ``fir`` / ``sos`` shortcuts and a reusable ``Plan``.  PyTorch supplies
device memory and the current CUDA stream; the filtering itself runs in the
CUDA library.  CPU tensors are accepted: ``tfx_chain_host`` copies channel
groups to the GPU, filters them and copies them back with the copies and the
filtering overlapped (pinned tensors let the copies run asynchronously).
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as N
from ._native import TfxError  # noqa: F401  (re-export)


def _stream_handle(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _check_signal(x: torch.Tensor) -> torch.Tensor:
    if x.dtype != torch.float32:
        raise TypeError("signal must be float32")
    if x.dim() == 1:
        x = x.unsqueeze(0)
    if x.dim() != 2:
        raise ValueError("signal must be [samples] or [channels, samples]")
    return x


def _row_stride(x: torch.Tensor) -> int:
    if x.size(1) > 1 and x.stride(1) != 1:
        raise ValueError("samples must be contiguous within each channel")
    if x.size(0) > 1:
        return x.stride(0)
    return max(1, x.size(1))


def chain(x: torch.Tensor, stages, out: torch.Tensor | None = None) -> torch.Tensor:
    """Apply ``stages`` (list of ("sos", rows[S x 6]) / ("fir", taps)) to every
    channel of ``x``.  ``out`` may be ``x`` (in place)."""
    squeeze = x.dim() == 1
    x2 = _check_signal(x)
    if not x2.is_cuda:
        y = _chain_host(x2, stages, out)
        return y[0] if squeeze and y.dim() == 2 and out is None else y
    if out is None:
        out2 = torch.empty_like(x2, memory_format=torch.contiguous_format)
        if x2.stride() != out2.stride():
            x2 = x2.contiguous()
    else:
        out2 = _check_signal(out)
        if out2.shape != x2.shape or out2.device != x2.device:
            raise ValueError("out must match x in shape and device")
        if out2.stride() != x2.stride():
            raise ValueError("out must have the same strides as x")
    C, Ns = x2.shape
    ld = _row_stride(x2)
    sl = N.StageList(stages)
    with torch.cuda.device(x2.device):
        rc = N.lib().tfx_chain(ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(out2.data_ptr()), C, Ns, ld,
                               sl.arr, sl.n, None, 0, _stream_handle(x2.device))
    N.check(rc, "tfx_chain")
    if out is not None:
        return out
    return out2[0] if squeeze else out2


def _chain_host(x: torch.Tensor, stages, out):
    """Host tensors: tfx_chain_host copies channel groups in, filters them and
    copies them out with the three overlapped (pinned buffers give overlap);
    returns once the result is in host memory."""
    if out is None:
        out = torch.empty(x.shape, dtype=torch.float32, pin_memory=x.is_pinned())
    out2 = _check_signal(out)
    if out2.is_cuda or out2.shape != x.shape:
        raise ValueError("out must be a host tensor of x's shape")
    if out2.stride() != x.stride():
        raise ValueError("out must have the same strides as x")
    C, Ns = x.shape
    ld = _row_stride(x)
    sl = N.StageList(stages)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    rc = N.lib().tfx_chain_host(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out2.data_ptr()), C, Ns, ld,
                                sl.arr, sl.n, ctypes.c_void_p(stream.cuda_stream))
    N.check(rc, "tfx_chain_host")
    stream.synchronize()
    return out


def fir(x: torch.Tensor, taps, out: torch.Tensor | None = None) -> torch.Tensor:
    """Causal FIR y[n] = sum_k h[k] x[n-k] on every channel (TorchFX Sec. 3)."""
    return chain(x, [("fir", taps)], out)


def sos(x: torch.Tensor, rows, out: torch.Tensor | None = None) -> torch.Tensor:
    """Cascade of second-order sections (rows b0 b1 b2 a0 a1 a2) on every channel."""
    return chain(x, [("sos", rows)], out)


class Plan:
    """A validated chain with its device constants, for repeated execution on
    buffers of one shape (no allocation or host synchronisation per call)."""

    def __init__(self, C: int, Nsamp: int, stages, ld: int | None = None, flags: int = 0,
                 device: int | None = None):
        self.C, self.N = int(C), int(Nsamp)
        self.ld = int(ld) if ld is not None else max(1, self.N)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._h = ctypes.c_void_p()
        sl = N.StageList(stages)
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_plan_create(ctypes.byref(self._h), self.C, self.N, self.ld, sl.arr, sl.n, flags)
        N.check(rc, "tfx_plan_create")
        self.workspace_size = int(N.lib().tfx_plan_workspace_size(self._h))
        self.launches_per_execute = int(N.lib().tfx_plan_launch_count(self._h))
        self._ws = None

    def workspace(self) -> torch.Tensor:
        if self._ws is None:
            self._ws = torch.empty(max(1, self.workspace_size), dtype=torch.uint8, device=self.device)
        return self._ws

    def _args(self, x, y, ws):
        x2 = _check_signal(x)
        y2 = _check_signal(y)
        for t in (x2, y2):
            if not t.is_cuda or tuple(t.shape) != (self.C, self.N):
                raise ValueError("buffers must be CUDA tensors of the plan's shape")
            if self.C > 1 and t.stride(0) != self.ld:
                raise ValueError("row stride differs from the plan's ld")
        w = self.workspace() if ws is None else ws
        return x2, y2, w

    def execute(self, x: torch.Tensor, y: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                plain: bool = False) -> torch.Tensor:
        if y is None:
            y = torch.empty_like(x)
        x2, y2, w = self._args(x, y, ws)
        fn = N.lib().tfx_plan_execute_plain if plain else N.lib().tfx_plan_execute
        with torch.cuda.device(self.device):
            rc = fn(self._h, ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(y2.data_ptr()),
                    ctypes.c_void_p(w.data_ptr()), w.numel(), _stream_handle(self.device))
        N.check(rc, "tfx_plan_execute_plain" if plain else "tfx_plan_execute")
        return y

    def get_error(self) -> int:
        with torch.cuda.device(self.device):
            return int(N.lib().tfx_plan_get_error(self._h))

    def close(self) -> None:
        if self._h:
            N.lib().tfx_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
