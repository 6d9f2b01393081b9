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


def assert_close_floored(got, ref, x, tol, what="", floor=1e-3):
    """The stated tolerance against each channel's output peak, floored at
    `floor` x the channel's input peak: a chain that attenuates by more than
    60 dB leaves an output that FP32 data (rounded relative to the input)
    cannot resolve to 1e-4 of its own peak."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    if got.ndim == 1:
        got, ref, x = got[None], ref[None], x[None]
    if got.shape[1] == 0:
        return 0.0
    err = np.max(np.abs(got - ref), axis=1)
    scale = np.maximum(np.max(np.abs(ref), axis=1), floor * np.max(np.abs(x), axis=1))
    rel = err / np.maximum(scale, 1e-30)
    worst = int(np.argmax(rel))
    assert np.all(rel <= tol), (f"{what}: channel {worst} max|err| {err[worst]:.3e} = {rel[worst]:.3e} x "
                                f"scale {scale[worst]:.3e} > tol {tol:g}")
    return float(rel.max())
