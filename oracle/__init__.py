"""FP64 CPU oracle for FIR / SOS filter chains -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never does, and this
package imports nothing from it.

The arithmetic lives in ``oracle.c`` (plain C, double precision):
  * ``sos``   -- cascade of second-order sections, each the literal DF-I
                 difference equation with zero initial state (TorchFX Sec. 3:
                 lfilter with user-supplied coefficients).
  * ``fir``   -- causal direct convolution, output length N (TorchFX Sec. 3,
                 Table 2 workload).
  * ``fir_at`` -- the same convolution at chosen output positions only.
  * ``chain`` -- stages applied in list order (TorchFX Sec. 3, pipe operator;
                 Table 4 workload).
  * ``chain_vjp`` -- gradients of sum(g * chain(x)) w.r.t. x and every
                 coefficient, from the chain's impulse response and from
                 forward-mode sensitivities of the difference equations
                 (the filters as layers inside a network, Sec. 3);
                 ``chain_vjp_dx_at`` gives dL/dx at chosen samples only.

Parity is pinned by closed forms and brute force in ``tests/test_oracle.py``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

FIR = 0
SOS = 1

_libs: dict = {}


class OracleLib:
    """ctypes view of one compiled oracle (the oracle, or a planted variant)."""

    def __init__(self, path: str):
        self.path = path
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        i32 = ctypes.c_int32
        lib.oracle_sos.argtypes = [dp, dp, i64, i64, dp, i32]
        lib.oracle_sos.restype = ctypes.c_int
        lib.oracle_fir.argtypes = [dp, dp, i64, i64, dp, i32]
        lib.oracle_fir.restype = ctypes.c_int
        lib.oracle_chain.argtypes = [dp, dp, i64, i64, ctypes.POINTER(i32),
                                     ctypes.POINTER(i32), ctypes.POINTER(dp), i32]
        lib.oracle_chain.restype = ctypes.c_int
        lib.oracle_chain_vjp.argtypes = [dp, dp, dp, dp, i64, i64, ctypes.POINTER(i32),
                                         ctypes.POINTER(i32), ctypes.POINTER(dp), i32]
        lib.oracle_chain_vjp.restype = ctypes.c_int
        lib.oracle_fir_at.argtypes = [dp, i64, dp, i32, ctypes.POINTER(i64), i64, dp]
        lib.oracle_fir_at.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_plant.restype = ctypes.c_int
        self.lib = lib

    @staticmethod
    def _dp(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    @staticmethod
    def _as_signal(x):
        x = np.asarray(x, dtype=np.float64)
        squeeze = x.ndim == 1
        x2 = np.ascontiguousarray(x.reshape(1, -1) if squeeze else x)
        if x2.ndim != 2:
            raise ValueError("signal must be [samples] or [channels, samples]")
        return x2, squeeze

    def sos(self, x, sos):
        x2, sq = self._as_signal(x)
        s = np.ascontiguousarray(np.asarray(sos, dtype=np.float64).reshape(-1, 6))
        y = np.empty_like(x2)
        rc = self.lib.oracle_sos(self._dp(x2), self._dp(y), x2.shape[0], x2.shape[1],
                                 self._dp(s), s.shape[0])
        if rc != 0:
            raise ValueError(f"oracle_sos failed ({rc})")
        return y[0] if sq else y

    def fir(self, x, h):
        x2, sq = self._as_signal(x)
        hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64).ravel())
        y = np.empty_like(x2)
        rc = self.lib.oracle_fir(self._dp(x2), self._dp(y), x2.shape[0], x2.shape[1],
                                 self._dp(hh), hh.size)
        if rc != 0:
            raise ValueError(f"oracle_fir failed ({rc})")
        return y[0] if sq else y

    def fir_at(self, x, h, idx):
        """Causal direct convolution of one channel x with taps h, evaluated
        only at the output positions idx (for signals too long to filter
        whole in the time a check may take)."""
        xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
        hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64).ravel())
        ii = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).ravel())
        out = np.empty(ii.size)
        rc = self.lib.oracle_fir_at(self._dp(xx), xx.size, self._dp(hh), hh.size,
                                    ii.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ii.size, self._dp(out))
        if rc != 0:
            raise ValueError(f"oracle_fir_at failed ({rc})")
        return out

    def chain(self, x, stages):
        """stages: list of ("fir", taps) or ("sos", [S x 6] rows)."""
        x2, sq = self._as_signal(x)
        kinds, counts, keep = [], [], []
        for kind, coef in stages:
            if kind == "fir":
                c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).ravel())
                kinds.append(FIR)
                counts.append(c.size)
            elif kind == "sos":
                c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1, 6))
                kinds.append(SOS)
                counts.append(c.shape[0])
            else:
                raise ValueError(f"unknown stage kind {kind!r}")
            keep.append(c)
        n = len(keep)
        ks = (ctypes.c_int32 * max(n, 1))(*kinds)
        cs = (ctypes.c_int32 * max(n, 1))(*counts)
        ptrs = (ctypes.POINTER(ctypes.c_double) * max(n, 1))(*[self._dp(c) for c in keep])
        y = np.empty_like(x2)
        rc = self.lib.oracle_chain(self._dp(x2), self._dp(y), x2.shape[0], x2.shape[1],
                                   ks, cs, ptrs, n)
        if rc != 0:
            raise ValueError(f"oracle_chain failed ({rc})")
        return y[0] if sq else y

    def chain_vjp(self, x, g, stages, want_dx: bool = True):
        """(dL/dx, [dL/dcoef per stage]) for upstream gradient g = dL/dy.
        With want_dx=False the O(N^2) input gradient is skipped (dL/dx None)."""
        x2, sq = self._as_signal(x)
        g2, _ = self._as_signal(g)
        if g2.shape != x2.shape:
            raise ValueError("g must match x")
        kinds, counts, keep = [], [], []
        for kind, coef in stages:
            if kind == "fir":
                c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).ravel())
                kinds.append(FIR)
                counts.append(c.size)
            else:
                c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1, 6))
                kinds.append(SOS)
                counts.append(c.shape[0])
            keep.append(c)
        n = len(keep)
        sizes = [c.size for c in keep]
        dcoef = np.zeros(max(1, sum(sizes)))
        ks = (ctypes.c_int32 * max(n, 1))(*kinds)
        cs = (ctypes.c_int32 * max(n, 1))(*counts)
        ptrs = (ctypes.POINTER(ctypes.c_double) * max(n, 1))(*[self._dp(c) for c in keep])
        dx = np.empty_like(x2) if want_dx else None
        rc = self.lib.oracle_chain_vjp(self._dp(x2), self._dp(g2), self._dp(dx) if want_dx else None,
                                       self._dp(dcoef),
                                       x2.shape[0], x2.shape[1], ks, cs, ptrs, n)
        if rc != 0:
            raise ValueError(f"oracle_chain_vjp failed ({rc})")
        grads, off = [], 0
        for c in keep:
            grads.append(dcoef[off:off + c.size].reshape(c.shape))
            off += c.size
        if dx is None:
            return None, grads
        return (dx[0] if sq else dx), grads

    def chain_vjp_dx_at(self, g, stages, idx):
        """dL/dx[m] of one channel at the sample indices idx, for long signals
        where the full O(N^2) input gradient is too slow: the chain is linear
        and time-invariant, so dL/dx[m] = sum_{n >= m} g[n] h[n - m] with h
        the chain's impulse response (computed by ``chain``)."""
        g = np.asarray(g, dtype=np.float64).ravel()
        N = g.size
        imp = np.zeros(N)
        if N:
            imp[0] = 1.0
        h = self.chain(imp, stages)
        return np.array([float(np.dot(g[m:], h[:N - m])) for m in idx])

    def num_threads(self) -> int:
        return int(self.lib.oracle_num_threads())

    def set_num_threads(self, n: int) -> None:
        self.lib.oracle_set_num_threads(int(n))


def load(plant: int = 0) -> OracleLib:
    """Build (if needed) and load the oracle; ``plant`` > 0 loads a variant with
    one deliberate mistake, used only to show the pins catch it."""
    if plant not in _libs:
        _libs[plant] = OracleLib(_build.build(plant))
    return _libs[plant]


def sos(x, sos_rows):
    return load().sos(x, sos_rows)


def fir(x, h):
    return load().fir(x, h)


def chain(x, stages):
    return load().chain(x, stages)


def fir_at(x, h, idx):
    return load().fir_at(x, h, idx)
