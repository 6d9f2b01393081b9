"""Reading R12 of the design (the whole chain as one FIR): a chain of SOS
cascades and FIRs is linear and time-invariant (TorchFX Sec. 3: the pipe
composes the stages), so it equals the causal convolution with its
composite impulse response h_c = g * f (g: the cascades' impulse response,
f: every FIR's taps convolved).  The plan truncates g at the first D with
sum_(n >= D) |g[n]| * sum|f| <= 1e-7 ||h_c||_2, which bounds the change of
every output by 1e-7 ||h_c||_2 max|x|.

Here D and h_c are derived in code of the test's own (g from the FP64
oracle run on an impulse), and the premise is checked against the oracle's
stage-by-stage result: the truncated composite reproduces it within the
stated bound, while a composite truncated at D/4 does not (so the check is
sensitive).  FP64 throughout; no GPU."""
import numpy as np

import oracle
from paper_2504_08624_gb300 import workloads as W


def _composite(stages, W_len=65536, eps=1e-7):
    lib = oracle.load()
    sos = [st for st in stages if st[0] == "sos"]
    imp = np.zeros(W_len)
    imp[0] = 1.0
    g = lib.chain(imp, sos)
    f = np.array([1.0])
    for k, c in stages:
        if k == "fir":
            f = np.convolve(f, np.asarray(c, dtype=np.float64))
    total = np.sum(np.abs(g))
    decayed = np.sum(np.abs(g[-4096:])) <= 1e-14 * total
    n2 = np.sqrt(np.sum(np.convolve(g[:16384], f)[:16384] ** 2))
    tail = np.cumsum(np.abs(g)[::-1])[::-1]  # tail[n] = sum_(k >= n) |g[k]|
    D = int(np.argmax(tail * np.sum(np.abs(f)) <= eps * n2))
    return g, f, D, n2, decayed


def _conv_causal(x, h):
    from numpy.fft import irfft, rfft
    n = x.shape[-1] + h.size - 1
    m = 1 << (n - 1).bit_length()
    return irfft(rfft(x, m) * rfft(h, m), m)[..., :x.shape[-1]]


def test_composite_matches_stage_by_stage_within_the_bound():
    wl = W.multichannel_fused()
    g, f, D, n2, decayed = _composite(wl.stages)
    assert decayed and 0 < D < 65536
    x = wl.make_signal(2, 60000).astype(np.float64)
    ref = oracle.chain(x, wl.stages)
    bound = 1e-7 * n2 * np.max(np.abs(x))
    y = _conv_causal(x, np.convolve(g[:D], f))
    err = np.max(np.abs(y - ref))
    # FP64 transform rounding adds ~1e-15 of the signal on top of the truncation
    assert err <= bound + 1e-13 * np.max(np.abs(ref)), (err, bound)
    # the composite cut at D/4 misses by far more: the criterion is not vacuous
    y4 = _conv_causal(x, np.convolve(g[:D // 4], f))
    assert np.max(np.abs(y4 - ref)) > 100 * bound


def test_composite_of_interleaved_stages():
    """Several cascades and FIRs interleaved: the order of LTI stages does not
    matter, so one composite (all sections, all FIRs) reproduces the chain."""
    stages = [("sos", W.butter_sos(4, 3000.0, W.FS)), ("fir", W.fir_lowpass(257, 9000.0, W.FS)),
              ("sos", W.random_peaking_bank(3, W.FS, 11)), ("fir", W.fir_highpass(101, 100.0, W.FS))]
    g, f, D, n2, decayed = _composite(stages)
    assert decayed
    x = W.white_uniform(2, 30000, 3).astype(np.float64)
    ref = oracle.chain(x, stages)
    y = _conv_causal(x, np.convolve(g[:D], f))
    bound = 1e-7 * n2 * np.max(np.abs(x))
    assert np.max(np.abs(y - ref)) <= bound + 1e-13 * np.max(np.abs(ref))


def test_slowly_decaying_cascade_is_not_composed():
    """A pole at radius 0.99999 has not decayed within 65536 samples: the
    reading does not apply (the plan keeps the chain's units)."""
    r, th = 0.99999, 0.3
    row = np.array([[1e-3, 0.0, -1e-3, 1.0, -2 * r * np.cos(th), r * r]])
    _, _, _, _, decayed = _composite([("sos", row), ("fir", W.fir_lowpass(101, 9000.0, W.FS))])
    assert not decayed
