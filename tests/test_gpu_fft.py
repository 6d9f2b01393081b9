"""FFT overlap-save FIR path (TFX_PLAN_FIR_FFT) against the FP64 oracle.

Block sizes: an L-tap FIR uses M = 2^m complex points (1024..16384) and
B = M - (L - 1) outputs per block, two blocks per CTA (real and imaginary
parts of one transform).  The cases cover one partial block, an odd block
count (the last CTA's second block is empty), lengths that end one sample
before / on / after a block boundary, channel counts that put the two blocks
of a CTA in different channels, in-place operation, padded strides, a cascade
ahead of the FFT unit, and the gradient of a trainable plan (the transposed
FIR runs on the same FFT unit).  Tolerance: 1e-5 of each channel's peak, as
for every FIR-only chain."""
import math

import numpy as np
import pytest

from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import assert_close, oracle_chain, tol_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _scheme(L, force=None):
    """(M, P) the plan's cost model picks (P = 0: single block): single-block
    30 + k_m M / B (B >= M/8), partitioned I_m + s_m P, fitted per m."""
    K = {10: 60.0, 11: 63.0, 12: 72.0, 13: 111.0, 14: 125.0}
    I = {10: 219.0, 11: 230.0, 12: 253.0, 13: 326.0, 14: 357.0}
    SP = {10: 20.0, 11: 21.4, 12: 23.6, 13: 24.7, 14: 26.0}
    best = None
    for m in range(10, 15):
        if force is not None and m != force:
            continue
        M = 1 << m
        B = M - (L - 1)
        if B >= M // 8:
            c = 30.0 + K[m] * M / B
            if best is None or c < best[0]:
                best = (c, M, 0)
        if m >= 11 or force == m:
            P = -(-L // (M // 2))
            c = I[m] + SP[m] * P
            if best is None or c < best[0]:
                best = (c, M, P)
    return best[1], best[2]


def _fft_block(L):
    """(M, B) of the single-block scheme the model picks for L."""
    M, P = _scheme(L)
    assert P == 0
    return M, M - (L - 1)


def run_fft(x, stages, inplace=False, ld=None, flags=0):
    from paper_2504_08624_gb300 import _native as N_
    from paper_2504_08624_gb300 import api
    C, Ns = x.shape
    ld = Ns if ld is None else ld
    buf = torch.zeros(C * ld + 8, dtype=torch.float32, device="cuda")
    xv = buf[:C * ld].view(C, ld)[:, :Ns]
    xv.copy_(torch.from_numpy(x))
    p = api.Plan(C, Ns, stages, ld=ld, flags=N_.TFX_PLAN_FIR_FFT | flags)
    y = xv if inplace else torch.zeros_like(buf)[:C * ld].view(C, ld)[:, :Ns]
    p.execute(xv, y)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    p.close()
    return y.cpu().numpy().astype(np.float64)


def check_fft(x, stages, tol=None, **kw):
    got = run_fft(x, stages, **kw)
    ref = oracle_chain(x, stages)
    return assert_close(got, ref, tol or tol_for(stages), str(kw))


def _taps(L, seed):
    return np.random.default_rng(seed).standard_normal(L) / math.sqrt(L)


@pytest.mark.parametrize("L", [64, 65, 129, 257, 335, 1025, 2049, 4097, 6146, 8193])
def test_fft_fir_lengths(L):
    """Forced FFT route (the model picks single-block for these lengths)."""
    M, B = _fft_block(L)
    for Ns in (1, B - 1, B, B + 1, 3 * B + 17):
        x = W.white_gauss(3, Ns, 31)
        check_fft(x, [("fir", _taps(L, L))])


@pytest.mark.parametrize("C", [1, 2, 5])
def test_fft_fir_blocks_across_channels(C):
    L = 1025
    M, B = _fft_block(L)
    x = W.pink(C, 2 * B + 300, 32)
    check_fft(x, [("fir", W.fir_lowpass(L, 4000.0, 48000.0))])


@pytest.mark.parametrize("inplace", [False, True])
def test_fft_fir_inplace_and_stride(inplace):
    x = W.white_gauss(3, 50000, 33)
    check_fft(x, [("fir", _taps(513, 5))], inplace=inplace, ld=50000 + 37)


@pytest.mark.parametrize("compose", [True, False])
def test_fft_fir_behind_cascade(compose):
    """Cascade then a long FIR: by default the whole chain is one FFT FIR of
    its composite response; with TFX_PLAN_NO_COMPOSE the cascade runs as its
    own unit, then the FFT unit."""
    from paper_2504_08624_gb300 import _native as N_
    wl = W.multichannel_fused()
    x = wl.make_signal(3, 40000)
    check_fft(x, wl.stages, wl.tol, flags=0 if compose else N_.TFX_PLAN_NO_COMPOSE)


def test_fft_fir_lowpass_and_bandpass():
    x = W.pink(2, 100000, 34)
    for h in (W.fir_lowpass(1025, 2000.0, 48000.0, ("kaiser", 8.0)),
              W.fir_bandpass(4097, 300.0, 3000.0, 48000.0, ("kaiser", 10.0)),
              W.fir_highpass(257, 8000.0, 48000.0)):
        check_fft(x, [("fir", h)])


def test_fft_fir_empty():
    from paper_2504_08624_gb300 import _native as N_
    from paper_2504_08624_gb300 import api
    for C, Ns in ((0, 100), (2, 0)):
        p = api.Plan(C, Ns, [("fir", _taps(300, 1))], flags=N_.TFX_PLAN_FIR_FFT)
        x = torch.zeros(C, Ns, device="cuda")
        y = torch.zeros_like(x)
        p.execute(x, y)
        torch.cuda.synchronize()
        p.close()


def _part_block(L):
    """(M, B, P) of the partitioned scheme the model picks for L."""
    M, P = _scheme(L)
    assert P > 0
    return M, M // 2, P


@pytest.mark.parametrize("L", [12290, 13000, 16384, 20000])
def test_partitioned_fir_lengths(L):
    """Beyond 12289 taps the FIR is partitioned: lengths shorter than one
    block, on and around block multiples, and an odd channel count (the last
    pair has no imaginary channel)."""
    M, B, P = _part_block(L)
    for C, Ns in ((3, 1), (3, B - 1), (2, B + 1), (3, 3 * B), (3, (P + 2) * B + 333)):
        x = W.white_gauss(C, Ns, 40)
        check_fft(x, [("fir", _taps(L, L))])


@pytest.mark.parametrize("m", [10, 11, 12, 13, 14])
def test_partitioned_every_transform_size(m):
    """Partitioned scheme at each forced transform size, P from 2 to 5."""
    from paper_2504_08624_gb300 import _native as N_
    M, B = 1 << m, (1 << m) // 2
    for L, C in ((M - M // 4 + 2, 3), (2 * M + 5, 4)):
        x = W.white_gauss(C, 4 * B + 19, 41)
        check_fft(x, [("fir", _taps(L, m + L))], flags=N_.TFX_PLAN_FIR_FFT_LOG(m))


@pytest.mark.parametrize("inplace", [False, True])
def test_partitioned_inplace_and_stride(inplace):
    x = W.white_gauss(5, 40000, 42)
    check_fft(x, [("fir", _taps(9000, 4))], inplace=inplace, ld=40000 + 9)


def test_partitioned_long_bandpass():
    """The 16384-tap Kaiser band-pass of the long-FIR workload, on its signal
    recipe, partitioned (and at each of the large transform sizes)."""
    from paper_2504_08624_gb300 import _native as N_
    wl = W.long_fir()
    x = wl.make_signal(3, 3 * 16384 + 1234)
    check_fft(x, wl.stages, 1e-5)
    for m in (12, 13, 14):
        check_fft(x, wl.stages, 1e-5, flags=N_.TFX_PLAN_FIR_FFT_LOG(m))


@pytest.mark.parametrize("m", [10, 11, 12, 13, 14])
def test_fft_fir_every_transform_size(m):
    """Each transform size (radix-4, -8, -16 and -2 first passes; 16384
    points with 512-thread CTAs of 32 points, radix 32, 32, 16) on a FIR it
    can hold, with a ragged tail."""
    from paper_2504_08624_gb300 import _native as N_
    L = (1 << m) // 4 + 1
    B = (1 << m) - (L - 1)
    x = W.white_gauss(3, 5 * B + 77, 38)
    check_fft(x, [("fir", _taps(L, m))], flags=N_.TFX_PLAN_FIR_FFT_LOG(m))
    x = W.white_gauss(2, 4 * B, 39)
    check_fft(x, [("fir", _taps(100, m))], flags=N_.TFX_PLAN_FIR_FFT_LOG(m))


@pytest.mark.parametrize("L", [257, 700, 7000])
def test_fft_fir_gradient_matches_oracle(L):
    """Trainable plan with the FFT flag: the input gradient's transposed FIR
    runs on the FFT unit; y, dx and every coefficient gradient against the
    oracle VJP."""
    from paper_2504_08624_gb300 import _native as N_
    from tests.test_gpu_grad import check_grad
    rows = W.random_stable_sos(2, 7, 0.3, 0.95)
    stages = [("sos", rows), ("fir", _taps(L, 3)), ("sos", W.random_stable_sos(1, 8, 0.3, 0.9))]
    x = W.white_gauss(3, 30000, 36)
    g = W.white_gauss(3, 30000, 37)
    check_grad(x, g, stages, flags=N_.TFX_PLAN_FIR_FFT)


def test_plan_describe_routes():
    """The plan description names each unit's route: the default sends a
    1025-tap FIR to the FFT, TFX_PLAN_FIR_TC keeps it on the tensor cores, a
    16384-tap FIR is partitioned, a short FIR behind a cascade stays fused."""
    from paper_2504_08624_gb300 import _native as N_
    from paper_2504_08624_gb300 import api
    wl = W.multichannel_fused()
    d = api.Plan(4, 100000, wl.stages).describe()
    assert [u["kind"] for u in d] == ["chain_fft"]
    assert d[0]["S"] == 8 and d[0]["L"] == 1025 and d[0]["Lc"] == d[0]["D"] + 1024
    assert d[0]["B"] == d[0]["M"] - (d[0]["Lc"] - 1)
    d = api.Plan(4, 100000, wl.stages, flags=N_.TFX_PLAN_NO_COMPOSE).describe()
    assert [u["kind"] for u in d] == ["cascade", "fir_fft"]
    assert d[0]["S"] == 8 and d[1]["L"] == 1025 and d[1]["P"] == 0 and d[1]["B"] == d[1]["M"] - 1024
    d = api.Plan(4, 100000, wl.stages, flags=N_.TFX_PLAN_FIR_TC).describe()
    assert [u["kind"] for u in d] == ["cascade", "fir_tc"] and d[1]["kernel"].startswith("k_fir_tc")
    d = api.Plan(2, 100000, W.long_fir().stages).describe()
    assert d[0]["kind"] == "fir_fft" and d[0]["P"] == -(-16384 // (d[0]["M"] // 2))
    d = api.Plan(2, 100000, [("sos", W.butter_sos(4, 1000.0, W.FS)), ("fir", _taps(31, 1))],
                 flags=N_.TFX_PLAN_NO_COMPOSE).describe()
    assert [u["kind"] for u in d] == ["fused"]
    # the FFT route is the default from 64 taps; shorter FIRs stay on the CUDA cores
    assert api.Plan(2, 100000, [("fir", _taps(64, 2))]).describe()[0]["kind"] == "fir_fft"
    assert api.Plan(2, 100000, [("fir", _taps(63, 2))]).describe()[0]["kind"] != "fir_fft"
    p = api.Plan(2, 100000, W.long_fir().stages)
    assert p.launches_per_execute == 2
    p.close()
