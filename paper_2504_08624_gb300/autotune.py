"""Autotuner for the batched launch.  It times candidate parameters on the
actual clips with CUDA events and caches the winners in a JSON file, so
that batches of the same kind skip the search.

Composed clips (each a whole chain run as one FFT FIR of its composite
response) are tuned per bucket of composite length, floor(log2(taps)): for
each bucket present, every transform size that holds the bucket's longest
response with at least a quarter of each transform as output (2^12, 2^13,
2^14 points) is timed on a sample of that bucket's clips, and the fastest is
kept (the batch then runs that bucket with it).  The clips that keep their
units are tuned as one group: the tensor-core FIR tile width (output blocks
of 128 per tile) and the tap count from which FIRs use the tensor cores
instead of the fused CUDA-core path.  Candidates the library rejects
(tables too large for the tile width) are skipped."""
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
FFT_SIZES = (10, 11, 12, 13, 14)
SAMPLE_SAMPLES = 30_000_000  # channel-samples timed per bucket and candidate


def default_cache_path() -> str:
    return os.environ.get("TFX_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tfx_autotune.json"))


def _bucket(v: float) -> int:
    return int(math.floor(math.log2(max(1.0, v))))


def signature(clips) -> str:
    """Bucketed description of a set of clips: histograms of log2 length,
    channels, sections and log2 taps, plus the clip count bucket."""
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


def _time_clips(clips, reps: int, **params) -> float:
    """Milliseconds per execution of a batch of `clips` with `params` (random
    input: the filters' cost does not depend on the values)."""
    b = api.Batch(clips, **params)
    x = torch.rand(max(1, b.total_samples), device=b.device) * 2 - 1
    y = b.empty()
    ms = _time(b, x, y, reps)
    if b.get_error() != 0:
        ms = float("inf")
    b.close()
    return ms


def _sample(clips, idx, budget: int):
    """Clips of `idx` in order until `budget` channel-samples."""
    out, n = [], 0
    for i in idx:
        out.append(clips[i])
        n += clips[i][0] * clips[i][1]
        if n >= budget:
            break
    return out


def _load(path, use_cache):
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def _store(path, cache):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)


def tune_batch(clips, x: torch.Tensor | None = None, cache_path: str | None = None, reps: int = 3,
               candidates=None, use_cache: bool = True) -> dict:
    """Best parameters for ``clips`` (list of (C, N, stages)).  Returns
    {"fir_nb", "tc_min_taps", "fft_m": {bucket: m}, "cached", "tried"};
    ``x`` (a packed input) is accepted for compatibility and not needed."""
    path = cache_path or default_cache_path()
    cache = _load(path, use_cache)
    tried = []
    all_cached = True
    # which clips compose, and their composite lengths (the cost model's plan)
    b0 = api.Batch(clips)
    info = [b0.clip_info(i) for i in range(len(clips))]
    b0.close()
    buckets = {}
    for i, (composed, taps, _) in enumerate(info):
        if composed:
            buckets.setdefault(_bucket(taps), []).append(i)
    fft_m = {}
    for k, idx in sorted(buckets.items()):
        key = f"fftm:L{k}"
        if use_cache and key in cache:
            fft_m[k] = int(cache[key])
            continue
        longest = max(info[i][1] for i in idx)
        sizes = [m for m in FFT_SIZES if longest - 1 <= (1 << m) - (1 << m) // 4]
        if len(sizes) < 2:
            continue
        all_cached = False
        sample = _sample(clips, idx, SAMPLE_SAMPLES)
        best = None
        for m in sizes:
            ms = _time_clips(sample, reps, fft_m={k: m})
            tried.append({"bucket": k, "fft_m": m, "clips": len(sample), "ms": ms})
            if best is None or ms < best[1]:
                best = (m, ms)
        fft_m[k] = best[0]
        cache[key] = best[0]
    # the clips that keep their units
    rest = [i for i, (composed, _, _) in enumerate(info) if not composed]
    tc = {"fir_nb": 128, "tc_min_taps": 64}
    if rest:
        sub = [clips[i] for i in rest]
        key = "units:" + signature(sub)
        if use_cache and key in cache:
            tc = {k: cache[key][k] for k in ("fir_nb", "tc_min_taps")}
        else:
            all_cached = False
            sample = _sample(clips, rest, SAMPLE_SAMPLES)
            best = None
            for cand in candidates or CANDIDATES:
                try:
                    ms = _time_clips(sample, reps, **cand)
                except TfxError:
                    tried.append({**cand, "ms": None})
                    continue
                tried.append({**cand, "ms": ms})
                if best is None or ms < best["ms"]:
                    best = {**cand, "ms": ms}
            if best is None:
                raise RuntimeError("no batch configuration could be built")
            tc = {"fir_nb": best["fir_nb"], "tc_min_taps": best["tc_min_taps"]}
            cache[key] = {**tc, "ms": best["ms"]}
    if use_cache and not all_cached:
        _store(path, cache)
    return {**tc, "fft_m": fft_m, "cached": all_cached, "tried": tried}
