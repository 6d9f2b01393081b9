"""Python API over libtfx: filter chains on [channels x samples] FP32 tensors.

TorchFX (arXiv 2504.08624, Sec. 3) applies FIR and IIR filters to every
channel of a signal and chains them with a pipe operator; this module exposes
the same operation: ``chain(x, stages)`` with stages applied in list order,
plus ``fir`` / ``sos`` shortcuts and a reusable ``Plan``.  PyTorch supplies
device memory and the current CUDA stream; the filtering itself runs in the
CUDA library.  CPU tensors are accepted: ``tfx_chain_host`` copies channel
groups to the GPU, filters them and copies them back with the copies and the
filtering overlapped (pinned tensors let the copies run asynchronously).

Gradients: ``chain_ad`` / ``FilterChain`` make the chain a differentiable
layer (Sec. 3 builds the filters as ``nn.Module`` classes for networks): the
forward keeps block-boundary states, the backward runs the library's
reverse-time adjoint kernels and returns dL/dx and dL/d(coefficients).
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

    def describe(self) -> list:
        """The plan's units in execution order, e.g.
        [{"kind": "cascade", "S": 8, "scan": "block", "carry": "fp32"},
         {"kind": "fir_fft", "L": 1025, "M": 4096, "B": 3072, "P": 0}]."""
        n = N.lib().tfx_plan_describe(self._h, None, 0)
        buf = ctypes.create_string_buffer(n + 1)
        N.lib().tfx_plan_describe(self._h, buf, n + 1)
        units = []
        for item in buf.value.decode().split(";") if n > 0 else []:
            kind, _, rest = item.partition(":")
            u = {"kind": kind}
            for kv in rest.split(","):
                k, _, v = kv.partition("=")
                u[k] = int(v) if v.lstrip("-").isdigit() else v
            units.append(u)
        return units

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

    # -- coefficient updates on the device ----------------------------------

    @property
    def sos_rows(self) -> int:
        return int(N.lib().tfx_plan_sos_rows(self._h))

    def update_sos(self, rows: torch.Tensor) -> None:
        """Recompute the plan's section constants on the GPU from ``rows`` (CUDA
        float64 [sos_rows x 6], every SOS row of the chain in order)."""
        if not rows.is_cuda or rows.dtype != torch.float64 or rows.numel() != 6 * self.sos_rows:
            raise ValueError("rows: CUDA float64 tensor of sos_rows x 6 values")
        rows = rows.contiguous()
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_plan_update_sos(self._h, ctypes.c_void_p(rows.data_ptr()), _stream_handle(self.device))
        N.check(rc, "tfx_plan_update_sos")
        # a composed chain falls back to its separate units after an update
        self.launches_per_execute = int(N.lib().tfx_plan_launch_count(self._h))

    def update_coefs(self, coef: torch.Tensor) -> None:
        """Set every coefficient of the chain from ``coef`` (CUDA float64,
        ``coef_count`` values in the layout of the backward's dcoef: stages in
        order, an FIR its taps, an SOS stage its raw rows) on the GPU, with no
        host round trip (tfx_plan_update_coefs)."""
        if not coef.is_cuda or coef.dtype != torch.float64 or coef.numel() != self.coef_count:
            raise ValueError("coef: CUDA float64 tensor of coef_count values")
        coef = coef.contiguous()
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_plan_update_coefs(self._h, ctypes.c_void_p(coef.data_ptr()), _stream_handle(self.device))
        N.check(rc, "tfx_plan_update_coefs")
        self.launches_per_execute = int(N.lib().tfx_plan_launch_count(self._h))

    # -- gradients (plans created with TFX_PLAN_TRAINABLE) -----------------

    @property
    def saved_size(self) -> int:
        return int(N.lib().tfx_plan_saved_size(self._h))

    @property
    def backward_workspace_size(self) -> int:
        return int(N.lib().tfx_plan_backward_workspace_size(self._h))

    @property
    def coef_count(self) -> int:
        return int(N.lib().tfx_plan_coef_count(self._h))

    @property
    def update_launches(self) -> int:
        """Kernels one update_coefs call launches (-1: the plan cannot be updated)."""
        return int(N.lib().tfx_plan_update_coefs_launch_count(self._h))

    def backward_launches(self, with_dx: bool = True, with_dcoef: bool = True) -> int:
        return int(N.lib().tfx_plan_backward_launch_count(self._h, int(with_dx), int(with_dcoef)))

    def new_saved(self) -> torch.Tensor:
        return torch.empty(max(1, self.saved_size), dtype=torch.uint8, device=self.device)

    def backward_workspace(self) -> torch.Tensor:
        if getattr(self, "_bws", None) is None:
            self._bws = torch.empty(max(1, self.backward_workspace_size), dtype=torch.uint8, device=self.device)
        return self._bws

    def forward_train(self, x: torch.Tensor, y: torch.Tensor, saved: torch.Tensor,
                      ws: torch.Tensor | None = None) -> torch.Tensor:
        x2, y2, w = self._args(x, y, ws)
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_plan_forward_train(self._h, ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(y2.data_ptr()),
                                                ctypes.c_void_p(saved.data_ptr()), saved.numel(),
                                                ctypes.c_void_p(w.data_ptr()), w.numel(), _stream_handle(self.device))
        N.check(rc, "tfx_plan_forward_train")
        return y

    def forward_train_mse(self, x: torch.Tensor, y: torch.Tensor, target: torch.Tensor, g: torch.Tensor,
                          loss: torch.Tensor, saved: torch.Tensor, ws: torch.Tensor | None = None) -> torch.Tensor:
        """Training forward with the MSE against ``target`` fused in
        (tfx_plan_forward_train_mse): fills y, saved, g = dL/dy and the
        device FP64 scalar ``loss``; returns loss."""
        x2, y2, w = self._args(x, y, ws)
        t2, g2, _ = self._args(target, g, ws)
        if not loss.is_cuda or loss.dtype != torch.float64 or loss.numel() < 1:
            raise ValueError("loss: CUDA float64 tensor")
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_plan_forward_train_mse(
                self._h, ctypes.c_void_p(x2.data_ptr()), ctypes.c_void_p(y2.data_ptr()),
                ctypes.c_void_p(t2.data_ptr()), ctypes.c_void_p(g2.data_ptr()),
                ctypes.cast(ctypes.c_void_p(loss.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                ctypes.c_void_p(saved.data_ptr()), saved.numel(), ctypes.c_void_p(w.data_ptr()), w.numel(),
                _stream_handle(self.device))
        N.check(rc, "tfx_plan_forward_train_mse")
        return loss

    @property
    def forward_train_mse_launches(self) -> int:
        return int(N.lib().tfx_plan_forward_train_mse_launch_count(self._h))

    def train_workspace(self) -> torch.Tensor:
        """A workspace large enough for both halves of a training step."""
        if getattr(self, "_tws", None) is None:
            n = max(1, self.workspace_size, self.backward_workspace_size)
            self._tws = torch.empty(n, dtype=torch.uint8, device=self.device)
        return self._tws

    def train_step_mse(self, x: torch.Tensor, y: torch.Tensor, target: torch.Tensor, g: torch.Tensor,
                       loss: torch.Tensor, dx: torch.Tensor | None, dcoef: torch.Tensor | None, saved: torch.Tensor,
                       ws: torch.Tensor | None = None) -> torch.Tensor:
        """One MSE training step (tfx_plan_train_step_mse): forward_train_mse
        then backward with its g, fused on a spectral plan; returns loss."""
        w = self.train_workspace() if ws is None else ws
        x2, y2, _ = self._args(x, y, w)
        t2, g2, _ = self._args(target, g, w)
        if dx is not None:
            self._args(dx, dx, w)
        if not loss.is_cuda or loss.dtype != torch.float64 or loss.numel() < 1:
            raise ValueError("loss: CUDA float64 tensor")
        if dcoef is not None and (dcoef.dtype != torch.float64 or not dcoef.is_cuda
                                  or dcoef.numel() < self.coef_count):
            raise ValueError("dcoef must be a CUDA float64 tensor of coef_count values")
        ptr = (lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None)
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_plan_train_step_mse(
                self._h, ptr(x2), ptr(y2), ptr(t2), ptr(g2),
                ctypes.cast(ctypes.c_void_p(loss.data_ptr()), ctypes.POINTER(ctypes.c_double)), ptr(dx),
                ctypes.cast(ptr(dcoef), ctypes.POINTER(ctypes.c_double)) if dcoef is not None else None,
                ctypes.c_void_p(saved.data_ptr()), saved.numel(), ctypes.c_void_p(w.data_ptr()), w.numel(),
                _stream_handle(self.device))
        N.check(rc, "tfx_plan_train_step_mse")
        return loss

    def train_step_launches(self, with_dx: bool = True, with_dcoef: bool = True) -> int:
        return int(N.lib().tfx_plan_train_step_mse_launch_count(self._h, int(with_dx), int(with_dcoef)))

    def backward(self, x: torch.Tensor, g: torch.Tensor, dx: torch.Tensor | None, dcoef: torch.Tensor | None,
                 saved: torch.Tensor, ws: torch.Tensor | None = None) -> None:
        x2, g2, _ = self._args(x, g, None)
        if dx is not None:
            self._args(dx, dx, None)
        if dcoef is not None and (dcoef.dtype != torch.float64 or not dcoef.is_cuda
                                  or dcoef.numel() < self.coef_count):
            raise ValueError("dcoef must be a CUDA float64 tensor of coef_count values")
        w = self.backward_workspace() if ws is None else ws
        ptr = (lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None)
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_plan_backward(self._h, ptr(x2), ptr(g2), ptr(dx), ptr(dcoef),
                                           ctypes.c_void_p(saved.data_ptr()), saved.numel(),
                                           ctypes.c_void_p(w.data_ptr()), w.numel(), _stream_handle(self.device))
        N.check(rc, "tfx_plan_backward")

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


def mse(y: torch.Tensor, target: torch.Tensor, g: torch.Tensor | None = None) -> torch.Tensor:
    """Mean squared error on the GPU: returns the loss (0-d float64 tensor) and,
    if ``g`` is given, writes dL/dy = 2 (y - target) / numel into it."""
    y2, t2 = _check_signal(y), _check_signal(target)
    if y2.shape != t2.shape or y2.stride() != t2.stride() or not y2.is_cuda:
        raise ValueError("y and target must be CUDA tensors of one shape and layout")
    if g is not None:
        g2 = _check_signal(g)
        if g2.shape != y2.shape or g2.stride() != y2.stride():
            raise ValueError("g must match y")
    loss = torch.empty((), dtype=torch.float64, device=y2.device)
    C, Ns = y2.shape
    with torch.cuda.device(y2.device):
        rc = N.lib().tfx_mse(ctypes.c_void_p(y2.data_ptr()), ctypes.c_void_p(t2.data_ptr()),
                             ctypes.c_void_p(g.data_ptr()) if g is not None else None, C, Ns, _row_stride(y2),
                             ctypes.c_void_p(loss.data_ptr()), _stream_handle(y2.device))
    N.check(rc, "tfx_mse")
    return loss


# ---------------------------------------------------------------------------
# autograd


class MSELossFunction(torch.autograd.Function):
    """mean((y - target)^2) with its gradient from the library's fused kernel
    (one pass computes the loss and dL/dy)."""

    @staticmethod
    def forward(ctx, y, target):
        y2 = _check_signal(y).contiguous()
        t2 = _check_signal(target).contiguous()
        g = torch.empty_like(y2)
        loss = mse(y2, t2, g)
        ctx.save_for_backward(g)
        ctx.shape = y.shape
        return loss

    @staticmethod
    def backward(ctx, gl):
        (g,) = ctx.saved_tensors
        return (g * gl.to(g.dtype)).reshape(ctx.shape), None


def mse_loss(y: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """Differentiable MSE on the GPU kernel (the differentiable-chain workload's loss)."""
    return MSELossFunction.apply(y, target)

# Trainable plans for ChainFunction, pooled by shape and chain structure
# (stage kinds and sizes), not by coefficient values: a training step updates
# a pooled plan's coefficients on the device (tfx_plan_update_coefs) instead
# of copying them to the host and building a new plan.  A plan is lent to
# one forward until its backward has run (its coefficients and saved state
# belong to that forward), so a pool holds as many plans as forwards are
# pending at once (one in a plain training loop).
_TRAIN_POOLS: dict = {}
_TRAIN_POOLS_MAX = 8   # structures kept
_TRAIN_POOL_PLANS = 4  # plans per structure


def _pool_key(C: int, Ns: int, device, coefs, kinds):
    return (C, Ns, str(device), tuple((k, tuple(c.shape)) for k, c in zip(kinds, coefs)))


def _release(plan: Plan) -> None:
    plan._pending = max(0, plan._pending - 1)
    if plan._pending == 0 and getattr(plan, "_evicted", False):
        plan.close()


def _lend_train_plan(C: int, Ns: int, device, kinds, coefs):
    """(plan, fresh): a pooled trainable plan with no pending backward, or a
    new one built from the current coefficient values (fresh = True)."""
    key = _pool_key(C, Ns, device, coefs, kinds)
    pool = _TRAIN_POOLS.pop(key, None)
    if pool is None:
        pool = []
        if len(_TRAIN_POOLS) >= _TRAIN_POOLS_MAX:
            old = _TRAIN_POOLS.pop(next(iter(_TRAIN_POOLS)))
            for q in old:  # closed now, or by the backward that still holds it
                q._evicted = True
                if q._pending == 0:
                    q.close()
    _TRAIN_POOLS[key] = pool  # most recent last
    for q in pool:
        if q._pending == 0:
            return q, False
    stages = [(k, c.detach().to("cpu", torch.float64).numpy()) for k, c in zip(kinds, coefs)]
    q = Plan(C, Ns, stages, flags=N.TFX_PLAN_TRAINABLE, device=device.index)
    q._pending = 0
    if len(pool) >= _TRAIN_POOL_PLANS:
        # more forwards pending than the pool keeps: the oldest idle-by-then plan is closed after its backward
        old = pool.pop(0)
        old._evicted = True
        if old._pending == 0:
            old.close()
    pool.append(q)
    return q, True


class ChainFunction(torch.autograd.Function):
    """y = chain(x) with gradients for x and every coefficient tensor.

    The plan comes from a pool keyed by shape and chain structure; its
    coefficients are set on the GPU from the coefficient tensors (one FP64
    concatenation and one update launch group), so a training loop with CUDA
    coefficient tensors makes no host round trip and allocates no plan after
    its first step.  Only a newly built plan reads the values on the host."""

    @staticmethod
    def forward(ctx, x, kinds, hold, *coefs):
        x2 = _check_signal(x).contiguous()
        if not x2.is_cuda:
            raise ValueError("chain_ad needs a CUDA signal")
        C, Ns = x2.shape
        plan, fresh = _lend_train_plan(C, Ns, x2.device, kinds, coefs)
        if not fresh:
            flat = torch.cat([c.detach().reshape(-1).to(device=x2.device, dtype=torch.float64) for c in coefs]) \
                if coefs else torch.zeros(0, dtype=torch.float64, device=x2.device)
            plan.update_coefs(flat)
        saved = plan.new_saved()
        y = torch.empty_like(x2)
        plan.forward_train(x2, y, saved)
        if hold:
            plan._pending += 1  # held until the backward has read the coefficients
        ctx.plan = plan
        ctx.meta = [(c.shape, c.dtype, c.device) for c in coefs]
        ctx.kinds = kinds
        ctx.squeeze = x.dim() == 1
        ctx.save_for_backward(x2, saved)
        return y[0] if ctx.squeeze else y

    @staticmethod
    def backward(ctx, gy):
        x2, saved = ctx.saved_tensors
        plan = ctx.plan
        try:
            g2 = _check_signal(gy.to(torch.float32)).contiguous()
            need_dx = ctx.needs_input_grad[0]
            need_dc = any(ctx.needs_input_grad[3:])
            if not (need_dx or need_dc):
                return (None, None, None) + (None,) * len(ctx.meta)
            dx = torch.empty_like(x2) if need_dx else None
            dcoef = torch.empty(max(1, plan.coef_count), dtype=torch.float64, device=x2.device) if need_dc else None
            plan.backward(x2, g2, dx, dcoef, saved)
        finally:
            _release(plan)
        grads, off = [], 0
        for (shape, dtype, device), need in zip(ctx.meta, ctx.needs_input_grad[3:]):
            n = 1
            for d in shape:
                n *= d
            if need and dcoef is not None:
                grads.append(dcoef[off:off + n].reshape(shape).to(device=device, dtype=dtype))
            else:
                grads.append(None)
            off += n
        if dx is not None and ctx.squeeze:
            dx = dx[0]
        return (dx, None, None, *grads)


def _chain_apply(x: torch.Tensor, kinds, coefs) -> torch.Tensor:
    """ChainFunction.apply, telling it whether a backward will follow (grad
    mode on and something requiring grad): only then does the forward keep
    its plan lent until that backward."""
    hold = torch.is_grad_enabled() and (x.requires_grad or any(c.requires_grad for c in coefs))
    return ChainFunction.apply(x, tuple(kinds), hold, *coefs)


def chain_ad(x: torch.Tensor, stages) -> torch.Tensor:
    """Differentiable chain: ``stages`` is a list of ("sos", rows [S x 6]) /
    ("fir", taps [L]) with torch tensors (any that require grad receive
    dL/d(coefficient); SOS rows as raw b0 b1 b2 a0 a1 a2)."""
    kinds = tuple(k for k, _ in stages)
    coefs = [c if torch.is_tensor(c) else torch.as_tensor(c, dtype=torch.float64) for _, c in stages]
    return _chain_apply(x, kinds, coefs)


class FilterChain(torch.nn.Module):
    """A chain of filters as an ``nn.Module`` with learnable coefficients
    (Sec. 3: the filters are modules that compose inside networks)."""

    def __init__(self, stages, learnable: bool = True):
        super().__init__()
        self.kinds = tuple(k for k, _ in stages)
        self.coefs = torch.nn.ParameterList(
            [torch.nn.Parameter(torch.as_tensor(c, dtype=torch.float64).clone(), requires_grad=learnable)
             for _, c in stages])

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        return _chain_apply(x, self.kinds, list(self.coefs))


class LearnableBiquadChain(torch.nn.Module):
    """The differentiable chain: a cascade of biquads whose poles are
    parameterised by radius r = rmin + rspan sigmoid(rho) and angle
    theta = pi sigmoid(phi) (stable for any parameter values), with free
    numerators, followed by a learnable FIR.  The SOS rows are built with torch
    ops, so autograd carries the chain rule from dL/d(rows) to rho and phi."""

    def __init__(self, rho, phi, b, h, rmin: float = 0.5, rspan: float = 0.49):
        super().__init__()
        f64 = dict(dtype=torch.float64)
        self.rho = torch.nn.Parameter(torch.as_tensor(rho, **f64).clone())
        self.phi = torch.nn.Parameter(torch.as_tensor(phi, **f64).clone())
        self.b = torch.nn.Parameter(torch.as_tensor(b, **f64).reshape(-1, 3).clone())
        self.h = torch.nn.Parameter(torch.as_tensor(h, **f64).clone())
        self.rmin, self.rspan = rmin, rspan

    def rows(self) -> torch.Tensor:
        r = self.rmin + self.rspan * torch.sigmoid(self.rho)
        th = torch.pi * torch.sigmoid(self.phi)
        ones = torch.ones_like(r)
        return torch.cat([self.b, torch.stack([ones, -2.0 * r * torch.cos(th), r * r], 1)], 1)

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        return _chain_apply(x, ("sos", "fir"), [self.rows(), self.h])


# ---------------------------------------------------------------------------
# batched launch over many clips


class Batch:
    """Many clips, each with its own (channels, samples, chain), filtered by a
    few batched launches over one packed input and one packed output buffer
    (``offsets[i]`` = first float of clip i; rows of its own length).
    ``params``: ``fir_nb`` (tensor-core FIR output blocks of 128 per tile),
    ``tc_min_taps`` (tensor cores from this many taps) and ``fft_m`` ({k: m}:
    composed clips whose composite response has floor(log2(taps)) = k use
    transforms of 2^m points), as picked by ``autotune.tune_batch``."""

    def __init__(self, clips, fir_nb: int = 128, tc_min_taps: int = 64, flags: int = 0,
                 device: int | None = None, fft_m: dict | None = None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.clips = [(int(C), int(Ns), list(st)) for C, Ns, st in clips]
        self._keep = [N.StageList(st) for _, _, st in self.clips]
        arr = (N.Clip * max(1, len(self.clips)))()
        for i, ((C, Ns, _), sl) in enumerate(zip(self.clips, self._keep)):
            arr[i].C, arr[i].N, arr[i].st, arr[i].nst = C, Ns, sl.arr, sl.n
        prm = N.BatchParams(flags, fir_nb, tc_min_taps)
        for k, m in (fft_m or {}).items():
            prm.fft_m[int(k)] = int(m)
        self.params = {"fir_nb": fir_nb, "tc_min_taps": tc_min_taps, "flags": flags,
                       "fft_m": {int(k): int(m) for k, m in (fft_m or {}).items()}}
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_batch_create(ctypes.byref(self._h), arr, len(self.clips), ctypes.byref(prm))
        N.check(rc, "tfx_batch_create")
        L = N.lib()
        self.total_samples = int(L.tfx_batch_total_samples(self._h))
        self.offsets = [int(L.tfx_batch_clip_offset(self._h, i)) for i in range(len(self.clips))]
        self.workspace_size = int(L.tfx_batch_workspace_size(self._h))
        self.launches_per_execute = int(L.tfx_batch_launch_count(self._h))
        self._ws = None

    def workspace(self) -> torch.Tensor:
        if self._ws is None:
            self._ws = torch.empty(max(1, self.workspace_size), dtype=torch.uint8, device=self.device)
        return self._ws

    def empty(self) -> torch.Tensor:
        return torch.empty(max(1, self.total_samples), dtype=torch.float32, device=self.device)

    def view(self, packed: torch.Tensor, i: int) -> torch.Tensor:
        """Clip i of a packed buffer as a [C, N] view."""
        C, Ns, _ = self.clips[i]
        o = self.offsets[i]
        return packed[o:o + C * Ns].view(C, Ns)

    def pack(self, signals) -> torch.Tensor:
        out = self.empty()
        for i, x in enumerate(signals):
            self.view(out, i).copy_(torch.as_tensor(x))
        return out

    def execute(self, x: torch.Tensor, y: torch.Tensor | None = None, ws: torch.Tensor | None = None):
        if y is None:
            y = self.empty()
        for t in (x, y):
            if not t.is_cuda or t.dtype != torch.float32 or t.numel() < self.total_samples or not t.is_contiguous():
                raise ValueError("packed buffers: contiguous float32 CUDA tensors of total_samples floats")
        w = self.workspace() if ws is None else ws
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_batch_execute(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                           ctypes.c_void_p(w.data_ptr()), w.numel(), _stream_handle(self.device))
        N.check(rc, "tfx_batch_execute")
        return y

    def clip_info(self, i: int) -> tuple:
        """(composed, composite taps, transform size exponent) of clip i."""
        c, t, m = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        N.check(N.lib().tfx_batch_clip_info(self._h, int(i), ctypes.byref(c), ctypes.byref(t), ctypes.byref(m)),
                "tfx_batch_clip_info")
        return bool(c.value), int(t.value), int(m.value)

    def groups(self) -> list:
        """[(kind, level, tiles, channel-samples, algorithmic flops)] per launch."""
        out = []
        for g in range(int(N.lib().tfx_batch_group_count(self._h))):
            k, lv = ctypes.c_int32(), ctypes.c_int32()
            t, sm, fl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
            N.check(N.lib().tfx_batch_group_info(self._h, g, ctypes.byref(k), ctypes.byref(lv), ctypes.byref(t),
                                                 ctypes.byref(sm), ctypes.byref(fl)), "tfx_batch_group_info")
            out.append((k.value, lv.value, t.value, sm.value, fl.value))
        return out

    def execute_group(self, g: int, x: torch.Tensor, y: torch.Tensor, ws: torch.Tensor | None = None) -> None:
        w = self.workspace() if ws is None else ws
        with torch.cuda.device(self.device):
            rc = N.lib().tfx_batch_execute_group(self._h, g, ctypes.c_void_p(x.data_ptr()),
                                                 ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                                 w.numel(), _stream_handle(self.device))
        N.check(rc, "tfx_batch_execute_group")

    def get_error(self) -> int:
        with torch.cuda.device(self.device):
            return int(N.lib().tfx_batch_get_error(self._h))

    def close(self) -> None:
        if self._h:
            N.lib().tfx_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# filter design on the GPU (FP64)


def design(specs, device=None) -> list:
    """Design filters on the GPU in FP64.  ``specs``: list of dicts with
    ``kind`` in butter_low / butter_high / cheby1_low (order, fc, fs[, ripple_db]),
    peaking (f0, Q, gain_db, fs), low_shelf / high_shelf (f0, gain_db, fs[, slope]),
    biquad_polar (rho, phi, b[, rmin, rspan]).  Returns one CUDA float64
    [sections x 6] tensor of raw rows per spec."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    arr = (N.Design * max(1, len(specs)))()
    counts = []
    for i, sp in enumerate(specs):
        d = arr[i]
        kind = sp["kind"]
        d.kind = N.DESIGN_KINDS[kind]
        d.fs = float(sp.get("fs", 48000.0))
        if kind in ("butter_low", "butter_high", "cheby1_low"):
            d.order, d.f1, d.p1 = int(sp["order"]), float(sp["fc"]), float(sp.get("ripple_db", 0.0))
        elif kind == "peaking":
            d.f1, d.p1, d.p2 = float(sp["f0"]), float(sp["Q"]), float(sp["gain_db"])
        elif kind in ("low_shelf", "high_shelf"):
            d.f1, d.p1, d.p2 = float(sp["f0"]), float(sp["gain_db"]), float(sp.get("slope", 1.0))
        elif kind == "biquad_polar":
            d.f1, d.f2 = float(sp.get("rmin", 0.5)), float(sp.get("rspan", 0.49))
            d.p1, d.p2 = float(sp["rho"]), float(sp["phi"])
            for j in range(3):
                d.b[j] = float(sp["b"][j])
        n = int(N.lib().tfx_design_sections(ctypes.byref(d)))
        if n < 0:
            raise ValueError(f"invalid design spec {sp}")
        counts.append(n)
    offs = [0]
    for n in counts:
        offs.append(offs[-1] + n)
    raw = ctypes.string_at(ctypes.addressof(arr), len(specs) * ctypes.sizeof(N.Design))
    dspecs = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev) if specs else torch.empty(1, dtype=torch.uint8, device=dev)
    doff = torch.tensor(offs[:-1] or [0], dtype=torch.int64, device=dev)
    rows = torch.empty(max(1, offs[-1]) * 6, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    with torch.cuda.device(dev):
        rc = N.lib().tfx_design_device(ctypes.c_void_p(dspecs.data_ptr()), len(specs), ctypes.c_void_p(doff.data_ptr()),
                                       ctypes.c_void_p(rows.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                       _stream_handle(dev))
    N.check(rc, "tfx_design_device")
    st = int(status.item())
    if st != 0:
        raise N.TfxError(st, "tfx_design_device")
    return [rows[6 * a:6 * b].view(b - a, 6) for a, b in zip(offs[:-1], offs[1:])]
