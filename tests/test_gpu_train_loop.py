"""A training loop through the public API (Sec. 3: filters as trainable
modules inside networks): SGD steps of LearnableBiquadChain on the GPU, each
step's coefficient gradients against the FP64 oracle's vector-Jacobian
product for that step's coefficients, with the plan kept and its
coefficients updated on the device (no new plan and no new device
allocation after the first step); device-side coefficient updates of a
forward plan (composed chain, FFT and CUDA-core FIRs, plain path);
gradient accumulation over two forwards before their backwards."""
import numpy as np
import pytest

import oracle
from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import assert_close, oracle_chain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _stage_errs(got_rows, got_h, grads):
    e_rows = np.max(np.abs(got_rows - grads[0])) / np.max(np.abs(grads[0]))
    e_h = np.max(np.abs(got_h - grads[1])) / np.max(np.abs(grads[1]))
    return e_rows, e_h


def test_sgd_steps_match_oracle_and_reuse_the_plan():
    from paper_2504_08624_gb300 import api
    wl = W.differentiable_chain_forward()
    pr = wl.meta["params"]
    C, Ns = 4, 12000
    x = torch.from_numpy(wl.make_signal(C, Ns)).cuda()
    target = api.chain(x, W.differentiable_chain_target())
    model = api.LearnableBiquadChain(pr["rho"], pr["phi"], pr["b"], pr["h"]).cuda()
    opt = torch.optim.SGD(model.parameters(), lr=0.05)
    before = {id(p) for pool in api._TRAIN_POOLS.values() for p in pool}
    plans, segs = [], []
    for step in range(3):
        opt.zero_grad(set_to_none=True)
        rows = model.rows()
        rows.retain_grad()
        y = api.chain_ad(x, [("sos", rows), ("fir", model.h)])
        loss = api.mse_loss(y, target)
        loss.backward()
        torch.cuda.synchronize()
        plans.extend(id(p) for pool in api._TRAIN_POOLS.values() for p in pool if id(p) not in before)
        # the oracle's VJP for this step's coefficients and dL/dy
        g = (2.0 * (y.detach().double() - target.double()) / (C * Ns)).cpu().numpy()
        stages = [("sos", rows.detach().cpu().numpy()), ("fir", model.h.detach().cpu().numpy())]
        _, grads = oracle.load().chain_vjp(x.double().cpu().numpy(), g, stages, want_dx=False)
        e_rows, e_h = _stage_errs(rows.grad.cpu().numpy(), model.h.grad.cpu().numpy(), grads)
        assert e_rows <= 1e-4 and e_h <= 1e-4, (step, e_rows, e_h)
        # the forward output against the oracle for the same coefficients
        assert_close(y.detach().cpu().numpy(), oracle_chain(x.cpu().numpy(), stages), 1e-4, f"step {step}")
        opt.step()
        segs.append(torch.cuda.memory_stats()["segment.all.allocated"])
    assert len(set(plans)) == 1, "a training step built a new plan"
    assert segs[2] == segs[1], "device memory was allocated after the first steps"


def test_gradient_accumulation_two_forwards_then_backwards():
    """Two forwards with different coefficients before either backward: each
    holds its own plan, so each backward sees its own coefficients."""
    from paper_2504_08624_gb300 import api
    wl = W.differentiable_chain_forward()
    C, Ns = 2, 8000
    x = torch.from_numpy(wl.make_signal(C, Ns)).cuda()
    rows1 = torch.from_numpy(np.asarray(wl.stages[0][1])).cuda().requires_grad_()
    h = torch.from_numpy(np.asarray(wl.stages[1][1], dtype=np.float64)).cuda().requires_grad_()
    rows2 = (rows1.detach() * torch.tensor([0.9, 1.1, 0.95, 1, 1, 1], dtype=torch.float64, device="cuda"))
    rows2.requires_grad_()
    y1 = api.chain_ad(x, [("sos", rows1), ("fir", h)])
    y2 = api.chain_ad(x, [("sos", rows2), ("fir", h)])
    g1 = torch.randn_like(y1)
    g2 = torch.randn_like(y2)
    y2.backward(g2)
    y1.backward(g1)
    torch.cuda.synchronize()
    lib = oracle.load()
    for rows, g in ((rows1, g1), (rows2, g2)):
        st = [("sos", rows.detach().cpu().numpy()), ("fir", h.detach().cpu().numpy())]
        _, grads = lib.chain_vjp(x.double().cpu().numpy(), g.double().cpu().numpy(), st, want_dx=False)
        e = np.max(np.abs(rows.grad.cpu().numpy() - grads[0])) / np.max(np.abs(grads[0]))
        assert e <= 1e-4, e


@pytest.mark.parametrize("flags", ["default", "no_compose", "cuda_cores"])
def test_update_coefs_forward_plan(flags):
    """A forward plan's coefficients replaced on the device: the multichannel
    chain (composed by default, which then runs its separate units; FFT FIR),
    the same with CUDA-core FIRs, and the plain path of the same plan."""
    from paper_2504_08624_gb300 import api, _native as N_
    fl = {"default": 0, "no_compose": N_.TFX_PLAN_NO_COMPOSE, "cuda_cores": N_.TFX_PLAN_FIR_CUDA_CORES}[flags]
    wl = W.multichannel_fused()
    C, Ns = 3, 60_000
    x = wl.make_signal(C, Ns)
    xt = torch.from_numpy(x).cuda()
    p = api.Plan(C, Ns, wl.stages, flags=fl)
    rng = np.random.default_rng(3)
    new = []
    for k, c in wl.stages:
        c = np.asarray(c, dtype=np.float64)
        if k == "sos":
            c = c.copy()
            c[:, :3] *= rng.uniform(0.5, 1.5, (c.shape[0], 1))
        else:
            c = c * rng.uniform(0.5, 1.5, c.shape)
        new.append((k, c))
    flat = torch.from_numpy(np.concatenate([c.ravel() for _, c in new])).cuda()
    p.update_coefs(flat)
    y = p.execute(xt)
    yp = p.execute(xt, plain=True)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    assert all(u["kind"] != "chain_fft" for u in p.describe())
    p.close()
    ref = oracle_chain(x, new)
    assert_close(y.cpu().numpy(), ref, 1e-4, f"{flags}: after update")
    assert_close(yp.cpu().numpy(), ref, 1e-4, f"{flags}: plain path after update")


@pytest.mark.parametrize("L", [7000, 16384])
def test_update_coefs_long_fft_firs(L):
    """FIR taps replaced on the device where the FFT unit uses 16384-point
    transforms (32 points per thread): single-block at 7000 taps, two
    partitions of 8192 taps at 16384; the spectra are rebuilt on the GPU by
    the same transform the filter runs."""
    from paper_2504_08624_gb300 import api
    h0 = W.fir_lowpass(L, 3000.0, W.FS)
    x = W.white_gauss(3, 3 * 16384 + 1234, 77)
    xt = torch.from_numpy(x).cuda()
    p = api.Plan(3, x.shape[1], [("fir", h0)])
    d = p.describe()
    assert d[0]["kind"] == "fir_fft" and d[0]["M"] == 16384 and (d[0]["P"] > 0) == (L > 12289), d
    h1 = h0 * np.random.default_rng(L).uniform(0.5, 1.5, L)
    p.update_coefs(torch.from_numpy(h1).cuda())
    y = p.execute(xt)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    p.close()
    assert_close(y.cpu().numpy(), oracle_chain(x, [("fir", h1)]), 1e-5, f"{L} taps after update")


def test_update_coefs_refused_for_tensor_core_firs():
    from paper_2504_08624_gb300 import api, _native as N_
    wl = W.multichannel_fused()
    p = api.Plan(2, 50_000, wl.stages, flags=N_.TFX_PLAN_FIR_TC)
    flat = torch.from_numpy(np.concatenate([np.asarray(c, dtype=np.float64).ravel() for _, c in wl.stages])).cuda()
    with pytest.raises(api.TfxError):
        p.update_coefs(flat)
    p.close()
