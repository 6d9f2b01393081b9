"""Gradients on the GPU (training forward + reverse-time adjoint backward)
against the FP64 oracle's vector-Jacobian product, through the C ABI.

The oracle computes dL/dx from the chain's impulse response and the
coefficient gradients from forward-mode sensitivities of the difference
equations; the GPU runs reverse-mode adjoint scans.  Tolerances (stated
against peaks because the signals are noise-like):
  * dL/dx: max|err| <= tol * peak|dL/dx| per channel, tol = 1e-4 once an IIR
    section is present and 1e-5 for FIR-only chains -- the forward's
    tolerances, since dL/dx is the same chain run over the reversed gradient;
  * coefficients: max|err| <= 1e-4 * max|grad| over each stage's
    coefficients (FP32 products summed per 1024-sample tile, then in FP64
    across tiles; the per-sample terms carry the forward's 1e-5-level
    relative error)."""
import numpy as np
import pytest

import oracle
from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import assert_close, tol_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COEF_TOL = 1e-4


def plan_for(C, N, stages, flags=0):
    from paper_2504_08624_gb300 import api, _native
    return api.Plan(C, N, stages, flags=_native.TFX_PLAN_TRAINABLE | flags)


def run_grad(x, g, stages, want_dx=True, want_dc=True, flags=0):
    """(y, dx, [dcoef per stage]) from forward_train + backward on the GPU."""
    C, N = x.shape
    p = plan_for(C, N, stages, flags)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    yd = torch.empty_like(xd)
    saved = p.new_saved()
    p.forward_train(xd, yd, saved)
    dx = torch.full_like(xd, float("nan")) if want_dx else None
    dc = torch.full((max(1, p.coef_count),), float("nan"), dtype=torch.float64, device="cuda") if want_dc else None
    p.backward(xd, gd, dx, dc, saved)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    p.close()
    grads = None
    if want_dc:
        dcn = dc.cpu().numpy()
        grads, off = [], 0
        for kind, c in stages:
            n = np.asarray(c).size
            grads.append(dcn[off:off + n].reshape(np.asarray(c).shape))
            off += n
    return (yd.cpu().numpy().astype(np.float64), None if dx is None else dx.cpu().numpy().astype(np.float64),
            grads)


def check_coefs(got, ref, stages, tol=COEF_TOL):
    worst = 0.0
    for i, ((kind, _), a, b) in enumerate(zip(stages, got, ref)):
        if b.size == 0:
            continue
        scale = np.max(np.abs(b))
        err = np.max(np.abs(a - b))
        assert np.all(np.isfinite(a)), f"stage {i} ({kind}): non-finite gradient"
        assert err <= tol * scale, f"stage {i} ({kind}): max|err| {err:.3e} > {tol:g} x {scale:.3e}"
        worst = max(worst, err / scale)
    return worst


def check_grad(x, g, stages, tol_dx=None, flags=0):
    y, dx, grads = run_grad(x, g, stages, flags=flags)
    lib = oracle.load()
    assert_close(y, lib.chain(x, stages), tol_for(stages), "training forward")
    dx_ref, grads_ref = lib.chain_vjp(x, g, stages)
    assert_close(dx, dx_ref, tol_dx or tol_for(stages), "dL/dx")
    check_coefs(grads, grads_ref, stages)


def a0_scaled(rows, seed):
    rng = np.random.default_rng(seed)
    return rows * rng.uniform(0.5, 2.0, (rows.shape[0], 1))


@pytest.mark.parametrize("N", [1, 2, 31, 32, 33, 1023, 1024, 1025, 3 * 1024 + 517])
def test_sos_grad_sizes(N):
    x = W.white_gauss(3, N, 5)
    g = W.white_gauss(3, N, 6)
    rows = a0_scaled(W.random_stable_sos(3, 17, 0.5, 0.99), 1)
    check_grad(x, g, [("sos", rows)])


@pytest.mark.parametrize("S", [1, 6, 8, 10, 17])
def test_sos_grad_sections(S):
    # more than 8 sections are split into several cascade units; long
    # cascades are peaking-EQ banks (gains near 1, zeros close to the poles)
    x = W.white_gauss(2, 5000, 7)
    g = W.white_gauss(2, 5000, 8)
    rows = W.random_stable_sos(S, 31 + S, 0.5, 0.95) if S <= 8 else W.random_peaking_bank(S, W.FS, 31 + S)
    check_grad(x, g, [("sos", rows)])


def test_sos_grad_long_signal():
    # 98 tiles per channel: long reverse look-back chains
    x = W.white_gauss(1, 100000, 9)
    g = W.white_gauss(1, 100000, 10)
    rows = W.random_stable_sos(2, 3, 0.9, 0.99)
    y, dx, grads = run_grad(x, g, [("sos", rows)])
    lib = oracle.load()
    idx = [0, 1, 1023, 1024, 50000, 99998, 99999]
    ref = lib.chain_vjp_dx_at(g[0], [("sos", rows)], idx)
    scale = np.max(np.abs(dx[0]))  # the channel's whole-signal peak
    assert np.max(np.abs(dx[0, idx] - ref)) <= 1e-4 * scale
    _, gref = lib.chain_vjp(x, g, [("sos", rows)], want_dx=False)
    check_coefs(grads, gref, [("sos", rows)])


@pytest.mark.parametrize("L", [1, 5, 17, 63, 64, 257, 385, 386, 1025])
def test_fir_grad(L):
    # input gradient: L < 64 CUDA-core FIR unit, L >= 64 tensor-core FIR over
    # the reversed gradient; tap gradient: the tensor-core correlation GEMM
    # (one lag window up to 385 taps, windows of 384 beyond)
    x = W.white_gauss(2, 6000, 11)
    g = W.white_gauss(2, 6000, 12)
    h = np.random.default_rng(L).normal(0.0, 1.0 / np.sqrt(L), L)
    check_grad(x, g, [("fir", h)])


@pytest.mark.parametrize("L", [5, 257, 700])
def test_fir_grad_cuda_cores(L):
    from paper_2504_08624_gb300 import _native
    x = W.white_gauss(3, 5000, 24)
    g = W.white_gauss(3, 5000, 25)
    h = np.random.default_rng(L + 1).normal(0.0, 1.0 / np.sqrt(L), L)
    check_grad(x, g, [("sos", W.random_stable_sos(2, 9, 0.5, 0.95)), ("fir", h)],
               flags=_native.TFX_PLAN_FIR_CUDA_CORES)


def test_fir_grad_channel_straddling_blocks():
    # N not a multiple of 128: 16-block K-steps of the tap-gradient GEMM span channels
    x = W.white_gauss(5, 1000, 26)
    g = W.white_gauss(5, 1000, 27)
    check_grad(x, g, [("fir", np.random.default_rng(3).normal(0, 0.1, 129))])


@pytest.mark.parametrize("name", ["sos_fir", "fir_sos", "sos_sos", "fir_fir", "empty_sos", "sos_fir_sos"])
def test_chain_grad(name):
    rng = np.random.default_rng(["sos_fir", "fir_sos", "sos_sos", "fir_fir", "empty_sos", "sos_fir_sos"].index(name))
    r1 = a0_scaled(W.random_stable_sos(2, 41, 0.5, 0.99), 2)
    r2 = W.random_stable_sos(3, 42, 0.5, 0.99)
    h1 = rng.normal(0, 0.1, 65)
    h2 = rng.normal(0, 0.3, 9)
    stages = {
        "sos_fir": [("sos", r1), ("fir", h1)],
        "fir_sos": [("fir", h2), ("sos", r1)],
        "sos_sos": [("sos", r1), ("sos", r2)],
        "fir_fir": [("fir", h1), ("fir", h2)],
        "empty_sos": [("sos", np.zeros((0, 6))), ("fir", h2)],
        "sos_fir_sos": [("sos", r2), ("fir", h1), ("sos", r1)],
    }[name]
    x = W.white_gauss(2, 4099, 13)
    g = W.white_gauss(2, 4099, 14)
    check_grad(x, g, stages)


def test_differentiable_chain_small():
    # the differentiable-chain workload's filters on a short signal
    w = W.differentiable_chain_forward()
    x = w.make_signal(4, 9000, 0)
    g = W.white_gauss(4, 9000, 15)
    check_grad(x, g, w.stages)


def test_grad_optional_outputs():
    stages = [("sos", W.random_stable_sos(2, 5, 0.5, 0.95)), ("fir", np.hanning(33))]
    x = W.white_gauss(2, 3000, 16)
    g = W.white_gauss(2, 3000, 17)
    _, dx_only, none = run_grad(x, g, stages, want_dx=True, want_dc=False)
    _, none2, dc_only = run_grad(x, g, stages, want_dx=False, want_dc=True)
    _, dx, dc = run_grad(x, g, stages)
    assert none is None and none2 is None
    assert np.array_equal(dx_only, dx)
    for a, b in zip(dc_only, dc):
        assert np.array_equal(a, b)


def test_grad_dx_may_alias_g():
    from paper_2504_08624_gb300 import api, _native  # noqa: F401
    stages = [("sos", W.random_stable_sos(2, 5, 0.5, 0.95)), ("fir", np.hanning(33))]
    x = W.white_gauss(2, 3000, 18)
    g = W.white_gauss(2, 3000, 19)
    p = plan_for(2, 3000, stages)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    saved = p.new_saved()
    p.forward_train(xd, torch.empty_like(xd), saved)
    ref = torch.empty_like(xd)
    p.backward(xd, gd, ref, None, saved)
    p.backward(xd, gd, gd, None, saved)
    torch.cuda.synchronize()
    assert torch.equal(ref, gd)
    p.close()


def test_grad_argument_errors():
    from paper_2504_08624_gb300 import api
    stages = [("sos", W.random_stable_sos(1, 5, 0.5, 0.95))]
    x = torch.randn(2, 100, device="cuda")
    plain = api.Plan(2, 100, stages)
    assert plain.saved_size == 0 and plain.backward_workspace_size == 0
    with pytest.raises(api.TfxError):
        plain.forward_train(x, torch.empty_like(x), torch.empty(256, dtype=torch.uint8, device="cuda"))
    p = plan_for(2, 100, stages)
    saved = p.new_saved()
    with pytest.raises(api.TfxError):  # in place: the backward needs x
        p.forward_train(x, x, saved)
    y = torch.empty_like(x)
    p.forward_train(x, y, saved)
    with pytest.raises(api.TfxError):  # saved buffer too small
        p.forward_train(x, y, saved[:16])
    with pytest.raises(api.TfxError):  # neither output requested
        p.backward(x, y, None, None, saved)
    with pytest.raises(api.TfxError):  # dx overlaps x
        p.backward(x, y, x, None, saved)
    torch.cuda.synchronize()
    p.close()
    plain.close()


def test_launch_counts():
    from paper_2504_08624_gb300 import _native
    stages = [("sos", W.random_stable_sos(6, 5, 0.5, 0.95)), ("fir", np.hanning(257))]
    p = plan_for(4, 5000, stages, _native.TFX_PLAN_NO_COMPOSE)  # the scan-adjoint route
    # cascade: adjoint scan + column sums + finalize; FIR: tap-gradient GEMM
    # (which also writes the reversed gradient) + column sums + FIR over the
    # reversed gradient; without coefficient gradients the FIR needs a flip
    assert p.backward_launches(True, True) == 3 + 3
    assert p.backward_launches(True, False) == 1 + 2
    assert p.launches_per_execute == 2
    p.close()


def test_zero_sizes():
    stages = [("sos", W.random_stable_sos(2, 5, 0.5, 0.95)), ("fir", np.hanning(9))]
    p = plan_for(0, 100, stages)
    dc = torch.full((p.coef_count,), 7.0, dtype=torch.float64, device="cuda")
    x = torch.empty(0, 100, device="cuda")
    p.forward_train(x, torch.empty_like(x), p.new_saved())
    p.backward(x, x, torch.empty_like(x), dc, p.new_saved())
    torch.cuda.synchronize()
    assert torch.all(dc == 0)
    p.close()


def test_chain_ad_autograd():
    from paper_2504_08624_gb300 import api
    w = W.differentiable_chain_forward()
    rows, h = w.stages[0][1], w.stages[1][1]
    x = w.make_signal(3, 7000, 0)
    g = W.white_gauss(3, 7000, 21)
    xt = torch.from_numpy(x.astype(np.float32)).cuda().requires_grad_(True)
    rt = torch.tensor(rows, dtype=torch.float64, requires_grad=True)
    ht = torch.tensor(h, dtype=torch.float64, device="cuda", requires_grad=True)
    y = api.chain_ad(xt, [("sos", rt), ("fir", ht)])
    y.backward(torch.from_numpy(g.astype(np.float32)).cuda())
    lib = oracle.load()
    dx_ref, (gr_ref, gh_ref) = lib.chain_vjp(x, g, w.stages)
    assert_close(xt.grad.cpu().numpy(), dx_ref, 1e-4, "autograd dL/dx")
    assert rt.grad.device.type == "cpu" and ht.grad.device.type == "cuda"
    check_coefs([rt.grad.numpy(), ht.grad.cpu().numpy()], [gr_ref, gh_ref], w.stages)


def test_fit_numerators_to_target():
    """Gradient steps on the MSE to a target-filtered signal lower the loss
    (the differentiable-chain workload's training step).  Only the section
    numerators and the FIR taps learn: the loss is then convex, and the
    poles cannot leave the unit circle."""
    from paper_2504_08624_gb300 import api
    rows = W.random_stable_sos(2, 77, 0.6, 0.8)
    h0 = np.zeros(17)
    h0[0] = 1.0
    target_rows = rows.copy()
    target_rows[:, :3] *= np.array([[1.3], [0.8]])
    h_t = h0.copy()
    h_t[3] = 0.4
    x = torch.from_numpy(W.white_gauss(4, 4096, 22).astype(np.float32)).cuda()
    target = api.chain(x, [("sos", target_rows), ("fir", h_t)])
    b = torch.nn.Parameter(torch.tensor(rows[:, :3]))
    a = torch.tensor(rows[:, 3:])
    fir = api.FilterChain([("fir", h0)])
    opt = torch.optim.Adam([b, *fir.parameters()], lr=0.02)
    losses = []
    for _ in range(80):
        opt.zero_grad()
        y = fir(api.chain_ad(x, [("sos", torch.cat([b, a], 1))]))
        loss = torch.mean((y - target) ** 2)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.05 * losses[0], losses[::10]


def test_mse_kernel():
    from paper_2504_08624_gb300 import api
    y = torch.randn(5, 3001, device="cuda")
    t = torch.randn(5, 3001, device="cuda")
    g = torch.empty_like(y)
    loss = api.mse(y, t, g)
    yn, tn = y.cpu().double().numpy(), t.cpu().double().numpy()
    ref = np.mean((yn - tn) ** 2)
    assert abs(float(loss) - ref) <= 1e-6 * ref
    assert np.max(np.abs(g.cpu().numpy() - 2 * (yn - tn) / yn.size)) <= 1e-6 * np.max(np.abs(2 * (yn - tn) / yn.size))


def test_differentiable_chain_full_size():
    """The full differentiable-chain workload (256 x 65,536, six biquads and a
    257-tap FIR) in the launch configuration the benchmark times: coefficient
    gradients against the oracle over all channels, dL/dx at sampled channels
    and samples (the full O(N^2) input gradient is out of the oracle's reach)."""
    w = W.differentiable_chain_forward()
    x = w.make_signal(w.C, w.N, 0)
    g = W.white_gauss(w.C, w.N, 23)
    y, dx, grads = run_grad(x, g, w.stages)
    lib = oracle.load()
    _, gref = lib.chain_vjp(x, g, w.stages, want_dx=False)
    check_coefs(grads, gref, w.stages)
    idx = [0, 1, 31, 32, 1023, 1024, 30000, 65534, 65535]
    for c in (0, 97, 255):
        ref = lib.chain_vjp_dx_at(g[c], w.stages, idx)
        got = dx[c, idx]
        # the sampled entries against the channel's whole-signal scale
        scale = np.max(np.abs(dx[c]))
        assert np.max(np.abs(got - ref)) <= 1e-4 * scale, (c, got, ref)
    ys = lib.chain(x[:2], w.stages)
    assert_close(y[:2], ys, 1e-4, "training forward")


def test_learnable_biquad_chain_parameter_grads():
    """Gradients w.r.t. the pole radius / angle parameters, numerators and FIR
    taps (autograd's chain rule on top of the adjoint kernels) against central
    differences of the FP64 oracle forward in those parameters."""
    from paper_2504_08624_gb300 import api
    p = W.differentiable_chain_params(41, n=3, taps=17)
    x = W.white_gauss(2, 3000, 30)
    g = W.white_gauss(2, 3000, 31)
    m = api.LearnableBiquadChain(p["rho"], p["phi"], p["b"], p["h"])
    y = m(torch.from_numpy(x.astype(np.float32)).cuda())
    y.backward(torch.from_numpy(g.astype(np.float32)).cuda())
    lib = oracle.load()

    def loss(pp):
        st = [("sos", W.biquad_rows(pp["rho"], pp["phi"], pp["b"])), ("fir", pp["h"])]
        return float(np.sum(g * lib.chain(x, st)))

    grads = {"rho": m.rho.grad.numpy(), "phi": m.phi.grad.numpy(), "b": m.b.grad.numpy(), "h": m.h.grad.numpy()}
    eps = 1e-6
    for name, idx in [("rho", 0), ("rho", 2), ("phi", 1), ("phi", 2), ("b", (1, 2)), ("b", (0, 0)), ("h", 3)]:
        pp = {k: np.array(v, dtype=np.float64) for k, v in p.items()}
        pm = {k: np.array(v, dtype=np.float64) for k, v in p.items()}
        pp[name][idx] += eps
        pm[name][idx] -= eps
        fd = (loss(pp) - loss(pm)) / (2 * eps)
        scale = np.max(np.abs(grads[name]))
        assert abs(grads[name][idx] - fd) <= 1e-4 * scale, (name, idx, grads[name][idx], fd)
