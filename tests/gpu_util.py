"""Helpers for the GPU parity tests: run a chain through the C ABI and compare
it with the FP64 oracle channel by channel."""
import numpy as np

import oracle


def per_channel_rel_err(got, ref):
    """max_n |got - ref| / max_n |ref| for each channel (TorchFX workloads are
    multichannel; the tolerance is stated against each channel's own peak)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.ndim == 1:
        got, ref = got[None], ref[None]
    err = np.max(np.abs(got - ref), axis=1) if got.shape[1] else np.zeros(got.shape[0])
    peak = np.max(np.abs(ref), axis=1) if ref.shape[1] else np.ones(ref.shape[0])
    return err / np.maximum(peak, 1e-30), err, peak


def assert_close(got, ref, tol, what=""):
    rel, err, peak = per_channel_rel_err(got, ref)
    worst = int(np.argmax(rel)) if rel.size else 0
    assert np.all(rel <= tol), (f"{what}: channel {worst} max|err| {err[worst]:.3e} = "
                                f"{rel[worst]:.3e} x peak {peak[worst]:.3e} > tol {tol:g}")
    return float(rel.max()) if rel.size else 0.0


def tol_for(stages):
    """1e-5 of the channel peak for FIR-only chains, 1e-4 once an IIR section
    is present (pole radius <= 0.999)."""
    return 1e-4 if any(k == "sos" and np.asarray(c).size for k, c in stages) else 1e-5


def oracle_chain(x, stages):
    return oracle.chain(np.asarray(x, dtype=np.float64), stages)


def assert_close_or_as_plain(got, ref, plain, tol, what="", factor=2.0):
    """The stated tolerance per channel against its own output peak, unfloored.

    Where the chain attenuates so strongly that an FP32 computation cannot
    resolve the output to `tol` of its own peak, the plain sequential FP32
    path (one thread per channel walking each section in time order, the
    comparison baseline) misses `tol` too; there the channel may not be more
    than `factor` times less accurate than that path.  Returns the per-channel
    errors of both (for the test's record)."""
    rel, err, peak = per_channel_rel_err(got, ref)
    rel_plain, _, _ = per_channel_rel_err(plain, ref)
    bad = [(c, rel[c], rel_plain[c]) for c in range(rel.size)
           if not (rel[c] <= tol or rel[c] <= factor * rel_plain[c])]
    assert not bad, (f"{what}: channel {bad[0][0]} error {bad[0][1]:.3e} of its peak exceeds tol {tol:g} and "
                     f"{factor:g} x the plain FP32 path's {bad[0][2]:.3e}")
    return rel, rel_plain
