"""Pipe-operator interface: ``result = signal | f1 | f2 | ...`` (TorchFX Sec. 3).

A :class:`Signal` holds a ``[channels x samples]`` float32 tensor and its
sample rate.  Filters hold their *design* parameters only; the sample rate
binds when a filter meets a signal (the paper's lazy binding), so the same
filter objects, or an ``nn.Sequential`` of them, can be piped into signals of
any rate.  Filters compose among themselves too: ``f1 | f2`` is a
:class:`Chain`.

GB300 difference from one-op-per-filter execution: piping records stages
instead of filtering.  ``signal | f1 | f2 | f3`` is a pending signal; the
whole chain runs as ONE fused library call (``api.chain``: the cascade and
FIR units of the plan, the signal crossing HBM once per unit) the first time
its samples are read (``.y``, ``.tensor()``, ``len``, or piping it into
something that needs them).  Every filter is also an ``nn.Module`` whose
``forward(x)`` applies it to a tensor at a fixed ``fs``.

Designs (host FP64, from ``workloads``): Butterworth and Chebyshev-I via the
bilinear transform, RBJ peaking and shelving biquads, windowed-sinc FIRs, and
raw SOS rows / FIR taps.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api
from . import workloads as W


class Filter(torch.nn.Module):
    """Base class: ``stages(fs)`` returns the library stages for sample rate fs."""

    fs: float | None = None

    def __init__(self, fs: float | None = None):
        super().__init__()
        self.fs = fs

    def stages(self, fs: float) -> list:  # pragma: no cover - abstract
        raise NotImplementedError

    def __or__(self, other) -> "Chain":
        return Chain([self, other])

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        if self.fs is None:
            raise ValueError(f"{type(self).__name__}: no sample rate bound; pipe a Signal into it "
                             "or construct it with fs=")
        return api.chain(x, self.stages(self.fs))


def _as_filters(f) -> list:
    if isinstance(f, Chain):
        return list(f.filters)
    if isinstance(f, Filter):
        return [f]
    if isinstance(f, torch.nn.Sequential):
        out = []
        for m in f:
            out.extend(_as_filters(m))
        return out
    raise TypeError(f"cannot pipe into {type(f).__name__}: expected a Filter, a Chain or an nn.Sequential of them")


class Chain(Filter):
    """Filters applied in order (the pipe operator between filters)."""

    def __init__(self, filters, fs: float | None = None):
        super().__init__(fs)
        flat = []
        for f in filters:
            flat.extend(_as_filters(f))
        self.filters = torch.nn.ModuleList(flat)

    def stages(self, fs: float) -> list:
        out = []
        for f in self.filters:
            out.extend(f.stages(fs))
        return out

    def __or__(self, other) -> "Chain":
        return Chain(list(self.filters) + _as_filters(other), self.fs)


class SOS(Filter):
    """Raw second-order sections (rows b0 b1 b2 a0 a1 a2)."""

    def __init__(self, rows, fs: float | None = None):
        super().__init__(fs)
        self.rows = np.asarray(rows, dtype=np.float64).reshape(-1, 6)

    def stages(self, fs):
        return [("sos", self.rows)]


class FIR(Filter):
    """Raw FIR taps."""

    def __init__(self, taps, fs: float | None = None):
        super().__init__(fs)
        self.taps = np.asarray(taps, dtype=np.float64).ravel()

    def stages(self, fs):
        return [("fir", self.taps)]


class Butterworth(Filter):
    """Butterworth low-/high-pass of the given order, -3 dB at fc."""

    def __init__(self, order: int, fc: float, btype: str = "low", fs: float | None = None):
        super().__init__(fs)
        self.order, self.fc, self.btype = order, fc, btype

    def stages(self, fs):
        return [("sos", W.butter_sos(self.order, self.fc, fs, self.btype))]


class Chebyshev1(Filter):
    """Chebyshev type-I low-pass; passband edge fc, ripple in dB."""

    def __init__(self, order: int, ripple_db: float, fc: float, fs: float | None = None):
        super().__init__(fs)
        self.order, self.ripple_db, self.fc = order, ripple_db, fc

    def stages(self, fs):
        return [("sos", W.cheby1_sos(self.order, self.ripple_db, self.fc, fs))]


class Peaking(Filter):
    """RBJ peaking EQ at f0 with quality Q and gain in dB."""

    def __init__(self, f0: float, Q: float, gain_db: float, fs: float | None = None):
        super().__init__(fs)
        self.f0, self.Q, self.gain_db = f0, Q, gain_db

    def stages(self, fs):
        return [("sos", W.peaking_sos(self.f0, self.Q, self.gain_db, fs))]


class LoShelving(Filter):
    """RBJ low shelf: gain_db below fc (default +6 dB), unity above."""

    def __init__(self, fc: float, gain_db: float = 6.0, slope: float = 1.0, fs: float | None = None):
        super().__init__(fs)
        self.fc, self.gain_db, self.slope = fc, gain_db, slope

    def stages(self, fs):
        return [("sos", W.shelving_sos("low", self.fc, self.gain_db, fs, self.slope))]


class HiShelving(Filter):
    """RBJ high shelf: gain_db above fc (default +6 dB), unity below."""

    def __init__(self, fc: float, gain_db: float = 6.0, slope: float = 1.0, fs: float | None = None):
        super().__init__(fs)
        self.fc, self.gain_db, self.slope = fc, gain_db, slope

    def stages(self, fs):
        return [("sos", W.shelving_sos("high", self.fc, self.gain_db, fs, self.slope))]


class WindowedSinc(Filter):
    """Windowed-sinc FIR: low-pass / high-pass at fc, or band-pass (fc = (f1, f2))."""

    def __init__(self, numtaps: int, fc, btype: str = "low", window="hamming", fs: float | None = None):
        super().__init__(fs)
        self.numtaps, self.fc, self.btype, self.window = numtaps, fc, btype, window

    def stages(self, fs):
        if self.btype == "low":
            h = W.fir_lowpass(self.numtaps, self.fc, fs, self.window)
        elif self.btype == "high":
            h = W.fir_highpass(self.numtaps, self.fc, fs, self.window)
        elif self.btype == "band":
            h = W.fir_bandpass(self.numtaps, self.fc[0], self.fc[1], fs, self.window)
        else:
            raise ValueError("btype must be 'low', 'high' or 'band'")
        return [("fir", h)]


class Signal:
    """A multichannel signal and its sample rate.  ``signal | filter`` returns a
    pending Signal; the recorded chain runs, fused, when the samples are read."""

    def __init__(self, y: torch.Tensor, fs: float):
        if not torch.is_tensor(y):
            y = torch.as_tensor(np.asarray(y, dtype=np.float32))
        self._y = y
        self.fs = float(fs)
        self._src = None      # pending: the input Signal's tensor
        self._stages = None   # pending: recorded stages

    @classmethod
    def _pending(cls, src: "Signal", stages: list) -> "Signal":
        s = cls.__new__(cls)
        s._y = None
        s.fs = src.fs
        if src._stages is not None:  # keep extending the same fused chain
            s._src, s._stages = src._src, src._stages + stages
        else:
            s._src, s._stages = src._y, list(stages)
        return s

    @property
    def pending_stages(self) -> int:
        """Stages recorded but not yet run (0 once materialised)."""
        return 0 if self._stages is None else len(self._stages)

    @property
    def y(self) -> torch.Tensor:
        if self._stages is not None:
            self._y = api.chain(self._src, self._stages)
            self._src, self._stages = None, None
        return self._y

    def tensor(self) -> torch.Tensor:
        return self.y

    def __len__(self) -> int:
        return self.y.shape[-1]

    def __or__(self, f) -> "Signal":
        return Signal._pending(self, Chain([f]).stages(self.fs))

    def __repr__(self) -> str:
        shape = tuple(self._y.shape) if self._y is not None else tuple(self._src.shape)
        return f"Signal(shape={shape}, fs={self.fs}, pending_stages={self.pending_stages})"
