"""Cascade on the tensor cores (k_sos_tc) against the FP64
oracle and against the CUDA-core look-back scan (TFX_PLAN_SCAN_LOOKBACK).

The route: blocks of 112 samples, zero-state responses and zero-start end
states by GEMM, a 16-dimensional scan of the block start states, their free
responses by a second GEMM; channels cut into segments (one persistent CTA
per SM walks its segments), every segment but a channel's first started D
samples early from zero state, its warm-up outputs discarded.  Cases: every section count up to 8,
poles up to radius 0.996 (D of several thousand samples), lengths ending
inside a block and a tile, single-segment and many-segment channels, loud
tiles next to quiet ones (per-tile scales), in-place operation and padded
strides.  Tolerance 1e-4 of each channel's peak."""
import numpy as np
import pytest

from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import assert_close, oracle_chain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE = 112 * 128


def _run(x, stages, flags=0, inplace=False, ld=None):
    """Through a plan that keeps its units (the tensor-core cascade is what
    these tests check, not the composed chain)."""
    from paper_2504_08624_gb300 import api, _native as N_
    flags |= N_.TFX_PLAN_NO_COMPOSE
    C, Ns = x.shape
    ld = Ns if ld is None else ld
    buf = torch.zeros(C * ld + 8, dtype=torch.float32, device="cuda")
    xv = buf[:C * ld].view(C, ld)[:, :Ns]
    xv.copy_(torch.from_numpy(x))
    p = api.Plan(C, Ns, stages, ld=ld, flags=flags)
    desc = p.describe()
    y = xv if inplace else torch.zeros_like(buf)[:C * ld].view(C, ld)[:, :Ns]
    p.execute(xv, y)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    p.close()
    return y.cpu().numpy().astype(np.float64), desc


def _check(x, stages, oracle_channels=None, min_segments=1, **kw):
    """oracle_channels: compare only these channels with the oracle (the
    channels are independent; long multichannel cases keep the oracle short)."""
    from paper_2504_08624_gb300 import _native as N_
    got, desc = _run(x, stages, **kw)
    assert desc[0]["kind"] == "cascade" and desc[0]["scan"] == "tc", desc
    assert desc[0]["segments"] >= min_segments, desc
    sel = slice(None) if oracle_channels is None else oracle_channels
    assert_close(got[sel], oracle_chain(x[sel], stages), 1e-4, str(kw))
    lb, d2 = _run(x, stages, flags=N_.TFX_PLAN_SCAN_LOOKBACK)
    assert d2[0]["scan"] == "block"
    assert_close(got, lb, 1e-4, "vs look-back scan")
    return desc[0]


@pytest.mark.parametrize("S", [1, 2, 3, 4, 5, 8])
def test_tc_cascade_sections(S):
    x = W.white_uniform(3, 3 * TILE + 1001, 50 + S)
    _check(x, [("sos", W.random_stable_sos(S, 60 + S, 0.3, 0.99))])


@pytest.mark.parametrize("N", [1, 111, 112, 113, TILE - 1, TILE, TILE + 1, 5 * TILE + 7777])
def test_tc_cascade_lengths(N):
    x = W.white_gauss(2, N, 51)
    _check(x, [("sos", W.butter_sos(4, 3000.0, W.FS))])


def test_tc_cascade_many_segments():
    """Few channels, long signal: each channel is cut into many segments, each
    but the first started D samples early (the multichannel workload's 8
    sections, poles to 0.996, D ~ 6000)."""
    wl = W.multichannel_fused()
    sos = [st for st in wl.stages if st[0] == "sos"]
    x = wl.make_signal(2, 3_000_000)
    d = _check(x, sos, min_segments=8)
    assert d["D"] >= 4096


def test_tc_cascade_multichannel_chain():
    """The multichannel workload's cascade on 16 channels of its recipe."""
    wl = W.multichannel_fused()
    sos = [st for st in wl.stages if st[0] == "sos"]
    x = wl.make_signal(16, 1_000_000)
    _check(x, sos, oracle_channels=slice(0, 16, 5))


def test_tc_cascade_loud_then_quiet():
    """Per-tile scales: tiles 1e4 louder next to near-silent ones (the carried
    state of a loud tile enters a quiet tile's free-response operand)."""
    rng = np.random.default_rng(54)
    N = 6 * TILE + 500
    x = rng.uniform(-1, 1, (2, N)).astype(np.float32)
    x[:, : 2 * TILE] *= 1e4
    x[:, 3 * TILE: 4 * TILE] *= 1e-4
    rows = W.random_stable_sos(4, 55, 0.5, 0.99)
    got, desc = _run(x, [("sos", rows)])
    assert desc[0]["scan"] == "tc"
    from paper_2504_08624_gb300 import api
    from tests.gpu_util import assert_close_or_as_plain
    p = api.Plan(x.shape[0], N, [("sos", rows)])
    xt = torch.from_numpy(x).cuda()
    plain = p.execute(xt, plain=True).cpu().numpy().astype(np.float64)
    p.close()
    assert_close_or_as_plain(got, oracle_chain(x, [("sos", rows)]), plain, 1e-4, "loud/quiet")


def test_tc_cascade_inplace_many_rounds():
    """In place, with more segments than CTAs (448 segments over the SMs, several
    rounds of the persistent walk): a segment's warm-up reads the preceding
    segment's input, which an in-place call must not see overwritten."""
    wl = W.multichannel_fused()
    sos = [st for st in wl.stages if st[0] == "sos"]
    x = wl.make_signal(64, 200_000)
    d = _check(x, sos, oracle_channels=slice(0, 64, 7), min_segments=4, inplace=True)
    assert d["D"] > 0, d


@pytest.mark.parametrize("inplace", [False, True])
@pytest.mark.parametrize("pad", [13, 4, 8])
def test_tc_cascade_inplace_and_stride(inplace, pad):
    """Row strides of N + pad floats: pad 8 keeps every row 32-byte aligned
    (one 32-byte load per 8-sample chunk), pad 4 alternates 32- and 16-byte
    aligned rows, pad 13 leaves rows 1 and 2 unaligned (scalar loads)."""
    x = W.white_uniform(3, 900_000, 52)
    _check(x, [("sos", W.random_peaking_bank(4, W.FS, 7))], inplace=inplace, ld=900_000 + pad)


def test_tc_cascade_then_fir():
    """Cascade on the tensor cores, then the FFT FIR unit (the headline chain's
    layout when its units stay separate)."""
    from paper_2504_08624_gb300 import _native as N_
    wl = W.multichannel_fused()
    x = wl.make_signal(16, 1_100_000)
    got, d = _run(x, wl.stages, flags=N_.TFX_PLAN_NO_COMPOSE)
    assert d[0]["scan"] == "tc" and d[1]["kind"] == "fir_fft", d
    assert_close(got[:2], oracle_chain(x[:2], wl.stages), wl.tol, "chain")


def test_tc_route_not_for_high_q_or_long_cascades():
    """Poles beyond 0.999 keep the FP64-carry warp scan, cascades of more than
    8 sections the look-back scan."""
    from paper_2504_08624_gb300 import api, _native as N_
    p = api.Plan(2, 100_000, [("sos", np.array([[1.0, 0.0, -1.0, 1.0, -1.9994, 0.9995]]))])
    assert p.describe()[0]["scan"] == "warp"
    p.close()
    # (kept from composing into one FFT FIR, which this decaying cascade would)
    p = api.Plan(2, 100_000, [("sos", W.random_stable_sos(9, 3, 0.3, 0.95))], flags=N_.TFX_PLAN_NO_COMPOSE)
    assert p.describe()[0]["scan"] == "block"
    p.close()
