"""Batched launch over many clips (each its own shape and chain) against the
FP64 oracle clip by clip, plus graph capture, argument errors and the
autotuner.  Tolerance per clip as for a single chain, against each channel's
own output peak: 1e-4 once an SOS stage is present, 1e-5 for FIR-only
chains.  Random chains can attenuate by well over 100 dB; where the plain
sequential FP32 path itself misses that tolerance on a channel (measured
beside, on the same input), the batched result may be at most twice as far
from the oracle as that path.  Every clip is also compared with the
single-clip library path (which the parity suite checks on its own) and the
per-channel errors are printed."""
import json

import numpy as np
import pytest

import oracle
from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import assert_close_or_as_plain, tol_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_clips():
    rng = np.random.default_rng(11)
    clips = []
    for i in range(14):
        C = int(rng.choice([1, 2, 3]))
        Ns = int(rng.integers(1, 40000))
        chain = W.random_chain(900 + i, max_sections=8, min_taps=33, max_taps=700)
        clips.append((C, Ns, chain))
    # fused short FIR, cascade only, FIR only, long FIR only, empty chain,
    # empty clip, zero channels, one sample
    clips.append((2, 9000, [("sos", W.random_stable_sos(3, 1, 0.5, 0.99)), ("fir", W.fir_lowpass(21, 4000.0, W.FS))]))
    clips.append((3, 12345, [("sos", W.random_stable_sos(5, 2, 0.5, 0.99))]))
    clips.append((1, 20000, [("fir", W.fir_lowpass(257, 3000.0, W.FS))]))
    clips.append((2, 30000, [("fir", W.fir_lowpass(2049, 3000.0, W.FS))]))
    clips.append((2, 500, []))
    clips.append((2, 0, [("sos", W.random_stable_sos(1, 3))]))
    clips.append((0, 100, [("sos", W.random_stable_sos(1, 3))]))
    clips.append((1, 1, [("sos", W.random_stable_sos(2, 4)), ("fir", np.hanning(101))]))
    clips.append((4, 70000, [("sos", W.random_stable_sos(8, 5, 0.3, 0.999)), ("sos", W.random_stable_sos(4, 6)),
                             ("fir", W.fir_lowpass(65, 9000.0, W.FS)), ("fir", W.fir_lowpass(33, 9000.0, W.FS))]))
    return clips


def run_batch(clips, **params):
    from paper_2504_08624_gb300 import api
    b = api.Batch(clips, **params)
    xs = [W.white_uniform(C, Ns, 50 + i) for i, (C, Ns, _) in enumerate(clips)]
    x = b.pack([torch.from_numpy(v) for v in xs])
    y = b.execute(x)
    torch.cuda.synchronize()
    assert b.get_error() == 0
    return b, xs, x, y


def _single_tc(xi, st, plain=False):
    """The single-clip path as an independent route: FIRs on the tensor cores
    (the batch and the default single-clip route send FIRs of 64+ taps to the
    FFT); with plain=True the plain sequential FP32 path of the same chain."""
    from paper_2504_08624_gb300 import _native as N_
    from paper_2504_08624_gb300 import api
    C, Ns = xi.shape
    p = api.Plan(C, Ns, st, flags=N_.TFX_PLAN_FIR_TC)
    xt = torch.from_numpy(xi).cuda()
    yt = torch.empty_like(xt)
    p.execute(xt, yt, plain=plain)
    torch.cuda.synchronize()
    p.close()
    return yt.cpu().numpy().astype(np.float64)


def check_clip(got, xi, st, what):
    """Per-channel errors of a batched clip against the oracle, next to the
    single-clip path's and the plain FP32 path's on the same input."""
    ref = oracle.chain(xi, st)
    plain = _single_tc(xi, st, plain=True) if st else xi
    single = _single_tc(xi, st) if st else xi
    tol = tol_for(st)
    rel, rel_plain = assert_close_or_as_plain(got, ref, plain, tol, what)
    rel_single, _ = assert_close_or_as_plain(single, ref, plain, tol, what + " (single-clip path)")
    print(f"{what}: max rel err batch {rel.max():.2e} single {rel_single.max():.2e} plain FP32 {rel_plain.max():.2e}"
          f" (tol {tol:g})")
    return rel, rel_plain


@pytest.mark.parametrize("params", [{}, {"fir_nb": 64, "flags": 1024}, {"fir_nb": 256, "tc_min_taps": 128, "flags": 1024},
                                    {"tc_min_taps": 32, "flags": 1024}, {"fft_m": {9: 13, 10: 14}}])
def test_batch_matches_oracle(params):
    clips = small_clips()
    from paper_2504_08624_gb300 import api
    b, xs, x, y = run_batch(clips, **params)
    for i, ((C, Ns, st), xi) in enumerate(zip(clips, xs)):
        if C == 0 or Ns == 0:
            continue
        got = b.view(y, i).cpu().numpy().astype(np.float64)
        check_clip(got, xi, st, f"clip {i} ({C}x{Ns})")
    b.close()


def test_batch_graph_capture_and_launch_count():
    from paper_2504_08624_gb300 import api
    clips = small_clips()
    b, xs, x, y = run_batch(clips)
    # a few batched launches, not one per clip (23 here): at most one per
    # (level, kernel, transform size) and one copy per empty-chain clip
    assert 1 <= b.launches_per_execute <= 12
    y2 = b.empty()
    ws = b.workspace()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.execute(x, y2, ws)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    y2.zero_()
    with torch.cuda.graph(g):
        b.execute(x, y2, ws)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y[:b.total_samples], y2[:b.total_samples])
    b.close()


def test_batch_argument_errors():
    from paper_2504_08624_gb300 import api, _native as N_
    clips = small_clips()[:3]
    # grouped units (composed clips need no workspace)
    b = api.Batch(clips, flags=N_.TFX_PLAN_NO_COMPOSE)
    assert b.workspace_size > 0
    x = b.empty()
    with pytest.raises(api.TfxError):  # in place is not allowed for batches
        b.execute(x, x)
    with pytest.raises(api.TfxError):  # workspace too small
        b.execute(x, b.empty(), torch.empty(16, dtype=torch.uint8, device="cuda"))
    with pytest.raises(api.TfxError):  # unstable section
        api.Batch([(1, 100, [("sos", [[1, 0, 0, 1, 0, 1.5]])])])
    b.close()


def test_autotuner_picks_and_caches(tmp_path):
    """Composed clips are tuned per composite-length bucket (transform size),
    the clips that keep their units as one group (tile width, tap threshold);
    a second call finds everything in the cache, and a batch built with the
    tuned parameters still matches the oracle."""
    from paper_2504_08624_gb300 import api, autotune
    clips = small_clips()[:10]
    # a clip whose cascade does not decay within the composition window (a
    # pole at radius 0.99999) keeps its units, with a FIR on the tensor cores
    r, th = 0.99999, 0.3
    slow = np.array([[1e-3, 0.0, -1e-3, 1.0, -2 * r * np.cos(th), r * r]])
    clips.append((2, 30000, [("sos", slow), ("fir", W.fir_lowpass(257, 9000.0, W.FS))]))
    path = str(tmp_path / "tune.json")
    cands = [{"fir_nb": 64, "tc_min_taps": 64}, {"fir_nb": 128, "tc_min_taps": 64}]
    r1 = autotune.tune_batch(clips, cache_path=path, reps=2, candidates=cands)
    assert not r1["cached"] and r1["tried"]
    assert {"fir_nb": r1["fir_nb"], "tc_min_taps": r1["tc_min_taps"]} in cands
    assert all(m in autotune.FFT_SIZES for m in r1["fft_m"].values())
    r2 = autotune.tune_batch(clips, cache_path=path, reps=2, candidates=cands)
    assert r2["cached"] and r2["fir_nb"] == r1["fir_nb"] and r2["fft_m"] == r1["fft_m"]
    b, xs, x, y = run_batch(clips, fir_nb=r1["fir_nb"], tc_min_taps=r1["tc_min_taps"], fft_m=r1["fft_m"])
    composed = [b.clip_info(i)[0] for i in range(len(clips))]
    assert any(composed) and not composed[-1]
    for i, ((C, Ns, st), xi) in enumerate(zip(clips, xs)):
        if C == 0 or Ns == 0:
            continue
        check_clip(b.view(y, i).cpu().numpy().astype(np.float64), xi, st, f"tuned clip {i}")
    b.close()


def test_batched_clips_workload_sampled():
    """The full 1000-clip workload in the configuration the benchmark times:
    every clip's data drawn on the GPU, then a sample of clips overwritten with
    their seeded host signals and compared with the oracle."""
    from paper_2504_08624_gb300 import api
    clips = W.batched_clips()
    spec = [(c.C, c.N, c.stages) for c in clips]
    b = api.Batch(spec)
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand(b.total_samples, device="cuda", generator=gen) * 2 - 1
    sample = [0, 1, 17, 333, 500, 998, 999]
    for i in sample:
        b.view(x, i).copy_(torch.from_numpy(clips[i].make_signal()))
    y = b.execute(x)
    torch.cuda.synchronize()
    assert b.get_error() == 0
    for i in sample:
        c = clips[i]
        got = b.view(y, i).cpu().numpy().astype(np.float64)
        # long clips: compare a prefix of the samples (the oracle is slow)
        n = min(c.N, 200000)
        xs = np.ascontiguousarray(c.make_signal()[:, :n])
        check_clip(got[:, :n], xs, c.stages, f"clip {i}")
    b.close()
