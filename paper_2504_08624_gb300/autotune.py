"""Autotuner for the batched launch: picks the tensor-core FIR tile width
(output blocks of 128 samples per tile) and the tap count from which FIRs
use the tensor cores instead of the fused CUDA-core path, by timing each
candidate on the actual batch with CUDA events, and caches the winner in a
JSON file keyed by the batch's bucketed signature (clip lengths, channel
counts, section counts, tap counts), so that batches of the same kind skip
the search.  Candidates that the library rejects (tables too large for the
tile width) are skipped."""
from __future__ import annotations

import hashlib
import json
import math
import os

import torch

from . import api
from ._native import TfxError

CANDIDATES = [
    {"fir_nb": nb, "tc_min_taps": t} for nb in (64, 128, 256) for t in (32, 64, 128)
]


def default_cache_path() -> str:
    return os.environ.get("TFX_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tfx_autotune.json"))


def _bucket(v: float) -> int:
    return int(math.floor(math.log2(max(1.0, v))))


def signature(clips) -> str:
    """Bucketed description of a batch: histograms of log2 length, channels,
    sections and log2 taps, plus the clip count bucket."""
    hist = {}
    for C, Ns, st in clips:
        S = sum(len(c) for k, c in st if k == "sos")
        L = sum(len(c) for k, c in st if k == "fir")
        key = f"n{_bucket(Ns)}c{C}s{S}l{_bucket(L)}"
        hist[key] = hist.get(key, 0) + 1
    body = json.dumps({"clips": _bucket(len(clips)), "h": sorted((k, _bucket(v)) for k, v in hist.items())})
    return hashlib.sha256(body.encode()).hexdigest()[:24]


def _time(batch: api.Batch, x: torch.Tensor, y: torch.Tensor, reps: int) -> float:
    batch.execute(x, y)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        batch.execute(x, y)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(clips, x: torch.Tensor, cache_path: str | None = None, reps: int = 3,
               candidates=None, use_cache: bool = True) -> dict:
    """Best parameters for ``clips`` (list of (C, N, stages)); ``x`` is a packed
    input for them.  Returns {"fir_nb", "tc_min_taps", "ms", "cached", "tried"}."""
    path = cache_path or default_cache_path()
    sig = signature(clips)
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and sig in cache:
        r = dict(cache[sig])
        r["cached"] = True
        return r
    best, tried = None, []
    y = None
    for cand in candidates or CANDIDATES:
        try:
            b = api.Batch(clips, **cand)
        except TfxError:
            tried.append({**cand, "ms": None})
            continue
        if y is None:
            y = b.empty()
        ms = _time(b, x, y, reps)
        if b.get_error() != 0:
            ms = float("inf")
        b.close()
        tried.append({**cand, "ms": ms})
        if best is None or ms < best["ms"]:
            best = {**cand, "ms": ms}
    if best is None:
        raise RuntimeError("no batch configuration could be built")
    best = {**best, "cached": False, "tried": tried}
    if use_cache:
        cache[sig] = {k: best[k] for k in ("fir_nb", "tc_min_taps", "ms")}
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return best
