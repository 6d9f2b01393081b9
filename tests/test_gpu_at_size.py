"""Parity at the benchmarked sizes, in the launch configuration the benchmark
times (the default plan of each workload): whole channels where the FP64
oracle finishes in seconds, sampled outputs where it does not.  Tolerances as
everywhere (per channel, against its own output peak): 1e-4 with SOS
stages, 1e-5 FIR-only; gradients 1e-4 of each stage's largest gradient."""
import numpy as np
import pytest

import oracle
from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import per_channel_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_multichannel_chain_full_size():
    """64 x 2,880,000 pink noise through the 8-section + 1025-tap chain; four
    whole channels (first, last, two inside) against the oracle."""
    from paper_2504_08624_gb300 import api
    wl = W.multichannel_fused()
    x = wl.make_signal()
    p = api.Plan(wl.C, wl.N, wl.stages)
    xt = torch.from_numpy(x).cuda()
    y = p.execute(xt)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    p.close()
    chs = [0, 21, 42, 63]
    got = y[chs].cpu().numpy().astype(np.float64)
    rel, _, _ = per_channel_rel_err(got, oracle.chain(x[chs].astype(np.float64), wl.stages))
    print("multichannel chain, per-channel max rel err:", " ".join(f"{v:.2e}" for v in rel))
    assert np.all(rel <= 1e-4), rel


def test_long_fir_full_length_sampled():
    """The 16384-tap band-pass over 8 channels of 4,194,304 samples (default
    route), checked at 544 sampled outputs per channel against the oracle's
    convolution at those positions; scale: the channel's largest |y|."""
    from paper_2504_08624_gb300 import api
    wl = W.long_fir()
    C = 8
    x = wl.make_signal(C, wl.N)
    h = np.asarray(wl.stages[0][1], dtype=np.float64)
    p = api.Plan(C, wl.N, wl.stages)
    y = p.execute(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert p.get_error() == 0
    p.close()
    idx = np.unique(np.concatenate([np.linspace(0, wl.N - 1, 512).astype(np.int64),
                                    np.linspace(0, h.size - 1, 32).astype(np.int64)]))
    lib = oracle.load()
    peak = y.abs().amax(dim=1).double().cpu().numpy()
    got = y[:, torch.from_numpy(idx).cuda()].double().cpu().numpy()
    for c in range(C):
        ref = lib.fir_at(x[c].astype(np.float64), h, idx)
        rel = np.max(np.abs(got[c] - ref)) / peak[c]
        assert rel <= 1e-5, (c, rel)


def test_differentiable_chain_full_size_step():
    """One training step of the 256 x 65,536 differentiable chain (training
    forward, MSE against the target chain, backward): the forward on four
    whole channels, dL/dx at sampled positions of the same channels, and the
    coefficient gradients of an 8-channel run against the oracle's VJP."""
    from paper_2504_08624_gb300 import api, _native as NAT
    wl = W.differentiable_chain_forward()
    x = torch.from_numpy(wl.make_signal()).cuda()
    target = api.chain(x, W.differentiable_chain_target())
    p = api.Plan(wl.C, wl.N, wl.stages, flags=NAT.TFX_PLAN_TRAINABLE)
    saved = p.new_saved()
    y = torch.empty_like(x)
    g = torch.empty_like(x)
    dx = torch.empty_like(x)
    dc = torch.empty(p.coef_count, dtype=torch.float64, device="cuda")
    p.forward_train(x, y, saved)
    api.mse(y, target, g)
    p.backward(x, g, dx, dc, saved)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    p.close()
    lib = oracle.load()
    chs = [0, 85, 170, 255]
    xs = x[chs].double().cpu().numpy()
    rel, _, _ = per_channel_rel_err(y[chs].double().cpu().numpy(), lib.chain(xs, wl.stages))
    assert np.all(rel <= 1e-4), rel
    idx = np.unique(np.concatenate([np.linspace(0, wl.N - 1, 48).astype(np.int64), np.arange(wl.N - 8, wl.N)]))
    gs = g[chs].double().cpu().numpy()
    dxs = dx[chs].double().cpu().numpy()
    for i in range(len(chs)):
        ref = lib.chain_vjp_dx_at(gs[i], wl.stages, idx)
        err = np.max(np.abs(dxs[i][idx] - ref)) / np.max(np.abs(dxs[i]))
        assert err <= 1e-4, (chs[i], err)
    # coefficient gradients: the same stages over the first 8 channels
    Cs = 8
    q = api.Plan(Cs, wl.N, wl.stages, flags=NAT.TFX_PLAN_TRAINABLE)
    x8, g8 = x[:Cs].contiguous(), g[:Cs].contiguous()
    sv = q.new_saved()
    q.forward_train(x8, torch.empty_like(x8), sv)
    dc8 = torch.empty(q.coef_count, dtype=torch.float64, device="cuda")
    q.backward(x8, g8, None, dc8, sv)
    torch.cuda.synchronize()
    assert q.get_error() == 0
    q.close()
    _, grads = lib.chain_vjp(x8.double().cpu().numpy(), g8.double().cpu().numpy(), wl.stages, want_dx=False)
    got = dc8.cpu().numpy()
    off = 0
    for gr in grads:
        ref = gr.ravel()
        err = np.max(np.abs(got[off:off + ref.size] - ref)) / np.max(np.abs(ref))
        assert err <= 1e-4, err
        off += ref.size
