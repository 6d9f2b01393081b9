"""The spectral training route on the GPU: a trainable chain that composes
runs its forward and input gradient as FFT FIRs of the chain's closed-form
spectrum and takes its coefficient gradients from the accumulated
gradient-input cross-spectrum.  Checked against the FP64 oracle's
vector-Jacobian product (dL/dx per channel at 1e-4 of its peak, the
forward's tolerance; coefficients at 1e-4 of each stage's largest gradient,
as for the scan route), against the scan-adjoint route of the same chain
(TFX_PLAN_NO_COMPOSE), and through device-side coefficient updates, including
the decay check that reports a response outgrowing the plan's overlap."""
import numpy as np
import pytest

import oracle
from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COEF_TOL = 1e-4


def chain(name):
    rng = np.random.default_rng(len(name))
    if name == "differentiable_chain":
        return W.differentiable_chain_forward().stages
    if name == "sos_only":
        return [("sos", W.random_stable_sos(4, 51, 0.5, 0.95))]
    if name == "fir_first":
        return [("fir", rng.normal(0, 0.2, 65)), ("sos", W.random_stable_sos(3, 52, 0.5, 0.9))]
    if name == "split_cascades":
        return [("sos", W.random_stable_sos(2, 53, 0.5, 0.9)), ("fir", W.fir_lowpass(129, 6000.0, W.FS)),
                ("sos", W.random_stable_sos(3, 54, 0.5, 0.9) * np.array([[2.0], [0.5], [1.0]]))]
    if name == "long_fir":
        return [("sos", W.random_stable_sos(2, 55, 0.5, 0.9)), ("fir", W.fir_lowpass(1025, 3000.0, W.FS))]
    if name == "sixteen_sections":  # two cascade units of the trainable plan
        return [("sos", W.random_stable_sos(16, 56, 0.5, 0.9))]
    raise ValueError(name)


def flat(stages):
    return np.concatenate([np.asarray(c, dtype=np.float64).ravel() for _, c in stages])


def grads(p, x, g, want_dx=True, want_dc=True, dx_into_g=False):
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    y = torch.empty_like(xd)
    saved = p.new_saved()
    p.forward_train(xd, y, saved)
    dx = (gd if dx_into_g else torch.full_like(xd, float("nan"))) if want_dx else None
    dc = torch.full((p.coef_count,), float("nan"), dtype=torch.float64, device="cuda") if want_dc else None
    p.backward(xd, gd, dx, dc, saved)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    return (y.cpu().numpy().astype(np.float64), None if dx is None else dx.cpu().numpy().astype(np.float64),
            None if dc is None else dc.cpu().numpy())


def split(dc, stages):
    out, off = [], 0
    for _, c in stages:
        n = np.asarray(c).size
        out.append(dc[off:off + n].reshape(np.asarray(c).shape))
        off += n
    return out


def check_coefs(got, ref, stages):
    worst = 0.0
    for i, ((kind, _), a, b) in enumerate(zip(stages, got, ref)):
        scale = np.max(np.abs(b))
        err = np.max(np.abs(a - b))
        assert np.all(np.isfinite(a)), f"stage {i} ({kind}): non-finite gradient"
        assert err <= COEF_TOL * scale, f"stage {i} ({kind}): max|err| {err:.3e} > {COEF_TOL:g} x {scale:.3e}"
        worst = max(worst, err / scale)
    return worst


def plan(C, N, stages, flags=0):
    from paper_2504_08624_gb300 import api, _native
    return api.Plan(C, N, stages, flags=_native.TFX_PLAN_TRAINABLE | flags)


@pytest.mark.parametrize("name,C,N", [("differentiable_chain", 4, 9000), ("sos_only", 3, 6001),
                                      ("fir_first", 2, 5000), ("split_cascades", 5, 12000),
                                      ("long_fir", 2, 20000), ("sixteen_sections", 2, 20000)])
def test_spectral_against_oracle(name, C, N):
    stages = chain(name)
    p = plan(C, N, stages)
    d = p.describe()
    assert [u["kind"] for u in d] == ["chain_spectral"], d
    assert p.saved_size == 0
    x = W.white_gauss(C, N, 60)
    g = W.white_gauss(C, N, 61)
    y, dx, dc = grads(p, x, g)
    p.close()
    lib = oracle.load()
    assert_close(y, lib.chain(x, stages), 1e-4, "training forward")
    dx_ref, gref = lib.chain_vjp(x, g, stages)
    assert_close(dx, dx_ref, 1e-4, "dL/dx")
    worst = check_coefs(split(dc, stages), gref, stages)
    print(f"{name}: {d[0]}, worst coefficient error {worst:.2e} of the stage's largest gradient")


def test_spectral_matches_scan_route():
    """The spectral and scan-adjoint routes of one chain agree to the
    oracle tolerances (each is checked against the oracle elsewhere)."""
    from paper_2504_08624_gb300 import _native
    stages = chain("differentiable_chain")
    C, N = 6, 20000
    x = W.white_gauss(C, N, 62)
    g = W.white_gauss(C, N, 63)
    ps, pn = plan(C, N, stages), plan(C, N, stages, _native.TFX_PLAN_NO_COMPOSE)
    assert ps.describe()[0]["kind"] == "chain_spectral" and pn.describe()[0]["kind"] != "chain_spectral"
    ys, dxs, dcs = grads(ps, x, g)
    yn, dxn, dcn = grads(pn, x, g)
    assert_close(ys, yn, 1e-4, "forward: spectral vs scan")
    assert_close(dxs, dxn, 1e-4, "dL/dx: spectral vs scan")
    check_coefs(split(dcs, stages), split(dcn, stages), stages)
    ps.close()
    pn.close()


def test_spectral_not_taken():
    """Chains outside the route keep the scan adjoint: two FIRs, more than
    16 sections, a pole above 0.999, a signal shorter than 2 (J + 1)."""
    h = W.fir_lowpass(65, 5000.0, W.FS)
    rows = W.random_stable_sos(2, 57, 0.5, 0.9)
    for stages, N in [([("sos", rows), ("fir", h), ("fir", h)], 20000),
                      ([("sos", W.random_stable_sos(17, 58, 0.5, 0.9))], 40000),
                      ([("sos", W.biquad_rows([0.0], [0.0], [[1.0, 0.0, 0.0]], rmin=0.9995, rspan=0.0))], 40000),
                      ([("sos", rows), ("fir", h)], 2000)]:
        p = plan(2, N, stages)
        assert all(u["kind"] != "chain_spectral" for u in p.describe()), p.describe()
        p.close()


def test_spectral_optional_outputs_and_alias():
    stages = chain("split_cascades")
    C, N = 3, 9000
    x = W.white_gauss(C, N, 64)
    g = W.white_gauss(C, N, 65)
    p = plan(C, N, stages)
    _, dx, dc = grads(p, x, g)
    _, dx_only, none = grads(p, x, g, want_dc=False)
    _, none2, dc_only = grads(p, x, g, want_dx=False)
    _, dx_alias, dc_alias = grads(p, x, g, dx_into_g=True)
    assert none is None and none2 is None
    assert np.array_equal(dx_only, dx) and np.array_equal(dx_alias, dx)
    assert np.array_equal(dc_only, dc) and np.array_equal(dc_alias, dc)
    p.close()


def test_spectral_launch_counts():
    stages = chain("differentiable_chain")
    p = plan(4, 9000, stages)
    # correlation, FP64 sum, section gradients, FIR tap gradient, a0 chain rule; dx: one FFT FIR
    assert p.backward_launches(True, True) == 6
    assert p.backward_launches(False, True) == 5
    assert p.backward_launches(True, False) == 1
    assert p.launches_per_execute == 1
    # section and tap writes, the FIR's spectrum, the chain's spectrum, the decay check
    assert p.update_launches == 5
    p.close()
    q = plan(3, 6001, chain("sos_only"))
    assert q.backward_launches(True, True) == 5 and q.update_launches == 3
    q.close()


def test_spectral_update_then_backward():
    """After tfx_plan_update_coefs the spectral plan follows the new
    coefficients (its chain spectrum is rebuilt on the device), matching the
    oracle and a plan built from them."""
    s0 = chain("split_cascades")
    s1 = [("sos", W.random_stable_sos(2, 73, 0.5, 0.9) * 1.7), ("fir", W.fir_lowpass(129, 9000.0, W.FS)),
          ("sos", W.random_stable_sos(3, 74, 0.5, 0.9))]
    C, N = 3, 15000
    x = W.white_gauss(C, N, 66)
    g = W.white_gauss(C, N, 67)
    p = plan(C, N, s0)
    p.update_coefs(torch.from_numpy(flat(s1)).cuda())
    assert p.describe()[0]["kind"] == "chain_spectral"
    y, dx, dc = grads(p, x, g)
    q = plan(C, N, s1)
    yq, dxq, dcq = grads(q, x, g)
    lib = oracle.load()
    assert_close(y, lib.chain(x, s1), 1e-4, "updated forward vs oracle")
    dx_ref, gref = lib.chain_vjp(x, g, s1)
    assert_close(dx, dx_ref, 1e-4, "updated dL/dx vs oracle")
    check_coefs(split(dc, s1), gref, s1)
    assert_close(y, yq, 1e-5, "updated vs fresh plan")
    assert_close(dx, dxq, 1e-5, "updated vs fresh plan dL/dx")
    # rows only (tfx_plan_update_sos): the FIR keeps its taps
    s2 = [("sos", s0[0][1]), ("fir", s1[1][1]), ("sos", s0[2][1])]
    p.update_sos(torch.from_numpy(np.vstack([s0[0][1], s0[2][1]])).cuda())
    y2, _, _ = grads(p, x, g, want_dc=False)
    assert_close(y2, lib.chain(x, s2), 1e-4, "rows-only update vs oracle")
    p.close()
    q.close()


def test_spectral_decay_check():
    """An update that moves a pole so close to the unit circle that the
    chain's response outlasts the overlap is reported as TFX_ERR_DECAY; a
    later update back inside clears nothing by itself (the status is read
    and cleared by get_error) and the plan computes correctly again."""
    s0 = chain("sos_only")
    C, N = 2, 8000
    p = plan(C, N, s0)
    J = p.describe()[0]["J"]
    assert J < 6144
    bad = s0[0][1].copy()
    bad[1] = W.biquad_rows([0.0], [-1.4], [[1.0, 0.5, 0.25]], rmin=0.999, rspan=0.0)[0]  # radius 0.999
    p.update_sos(torch.from_numpy(bad).cuda())
    torch.cuda.synchronize()
    assert p.get_error() == -8  # TFX_ERR_DECAY
    p.update_sos(torch.from_numpy(s0[0][1]).cuda())
    torch.cuda.synchronize()
    assert p.get_error() == 0
    x = W.white_gauss(C, N, 68)
    g = W.white_gauss(C, N, 69)
    y, dx, dc = grads(p, x, g)
    lib = oracle.load()
    assert_close(y, lib.chain(x, s0), 1e-4, "after the decay error")
    p.close()


def test_spectral_full_size_differentiable_chain():
    """The bench's training configuration (256 x 65,536) on the spectral
    route: coefficient gradients against the oracle over all channels,
    dL/dx at sampled channels and samples."""
    w = W.differentiable_chain_forward()
    p = plan(w.C, w.N, w.stages)
    assert p.describe()[0]["kind"] == "chain_spectral"
    x = w.make_signal(w.C, w.N, 0)
    g = W.white_gauss(w.C, w.N, 23)
    y, dx, dc = grads(p, x, g)
    p.close()
    lib = oracle.load()
    _, gref = lib.chain_vjp(x, g, w.stages, want_dx=False)
    worst = check_coefs(split(dc, w.stages), gref, w.stages)
    idx = [0, 1, 1023, 1024, 30000, 65534, 65535]
    for c in (0, 131, 255):
        ref = lib.chain_vjp_dx_at(g[c], w.stages, idx)
        assert np.max(np.abs(dx[c, idx] - ref)) <= 1e-4 * np.max(np.abs(dx[c])), c
    assert_close(y[:2], lib.chain(x[:2], w.stages), 1e-4, "training forward")
    print(f"full-size spectral gradients: worst {worst:.2e} of the stage's largest gradient")


@pytest.mark.parametrize("route", ["spectral", "units"])
def test_forward_train_mse_fused(route):
    """tfx_plan_forward_train_mse equals tfx_plan_forward_train followed by
    tfx_mse: y and g bit for bit, the loss to FP64 summation order; g may
    replace the target; the backward from the fused g is the same."""
    from paper_2504_08624_gb300 import api, _native
    stages = chain("differentiable_chain")
    C, N = 5, 20000
    p = plan(C, N, stages, 0 if route == "spectral" else _native.TFX_PLAN_NO_COMPOSE)
    assert (p.describe()[0]["kind"] == "chain_spectral") == (route == "spectral")
    assert p.forward_train_mse_launches == (1 if route == "spectral" else p.launches_per_execute + 1)
    x = torch.from_numpy(W.white_gauss(C, N, 70).astype(np.float32)).cuda()
    tgt = torch.from_numpy(W.white_gauss(C, N, 71).astype(np.float32)).cuda()
    saved = p.new_saved()
    y1, g1 = torch.empty_like(x), torch.empty_like(x)
    p.forward_train(x, y1, saved)
    l1 = api.mse(y1, tgt, g1)
    y2, g2 = torch.full_like(x, float("nan")), torch.full_like(x, float("nan"))
    l2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    saved2 = p.new_saved()
    p.forward_train_mse(x, y2, tgt, g2, l2, saved2)
    t3 = tgt.clone()
    y3 = torch.empty_like(x)
    l3 = torch.empty(1, dtype=torch.float64, device="cuda")
    p.forward_train_mse(x, y3, t3, t3, l3, p.new_saved())  # g replaces the target
    torch.cuda.synchronize()
    assert p.get_error() == 0
    assert torch.equal(y1, y2) and torch.equal(g1, g2) and torch.equal(y1, y3) and torch.equal(g1, t3)
    assert abs(float(l2) - float(l1)) <= 1e-6 * abs(float(l1)) and abs(float(l3) - float(l1)) <= 1e-6 * abs(float(l1))
    dc1 = torch.empty(p.coef_count, dtype=torch.float64, device="cuda")
    dc2 = torch.empty_like(dc1)
    p.backward(x, g1, None, dc1, saved)
    p.backward(x, g2, None, dc2, saved2)
    torch.cuda.synchronize()
    assert torch.equal(dc1, dc2)
    with pytest.raises(api.TfxError):  # the target may not overlap y
        p.forward_train_mse(x, y2, y2, g2, l2, saved2)
    p.close()


@pytest.mark.parametrize("case", ["differentiable_chain", "odd_blocks", "8192_points", "units"])
def test_train_step_mse(case):
    """tfx_plan_train_step_mse against tfx_plan_forward_train_mse followed by
    tfx_plan_backward on the same inputs: y, g and dL/dx bit for bit, the
    loss to FP64 summation order, the coefficient gradients to FP32 rounding
    (the fused correlation pairs other blocks as real and imaginary parts)
    and against the oracle's vector-Jacobian product of the step's own g;
    dx taking g's place and no dx give the same gradients; the launch count.
    odd_blocks: an odd number of blocks in all (the last pair has no second
    block) and pairs that straddle two channels.  units: a plan kept on its
    units runs the two calls in order."""
    from paper_2504_08624_gb300 import _native
    if case == "8192_points":
        stages = [("sos", W.random_stable_sos(4, 82, 0.9, 0.99)), ("fir", W.fir_lowpass(1025, 3000.0, W.FS))]
        C, N = 3, 30000
    else:
        stages = chain("differentiable_chain")
        C, N = {"differentiable_chain": (4, 20000), "odd_blocks": (5, 12345), "units": (4, 9000)}[case]
    p = plan(C, N, stages, _native.TFX_PLAN_NO_COMPOSE if case == "units" else 0)
    d = p.describe()[0]
    spectral = d["kind"] == "chain_spectral"
    assert spectral == (case != "units"), d
    if case == "odd_blocks":
        assert (C * -(-N // d["B"])) % 2 == 1, d
    xn, tn = W.white_gauss(C, N, 90), W.white_gauss(C, N, 91)
    x = torch.from_numpy(xn.astype(np.float32)).cuda()
    tgt = torch.from_numpy(tn.astype(np.float32)).cuda()

    def scalar():
        return torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")

    def coefs():
        return torch.full((p.coef_count,), float("nan"), dtype=torch.float64, device="cuda")

    y1, g1, dx1, l1, dc1 = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x), scalar(), coefs()
    s1 = p.new_saved()
    p.forward_train_mse(x, y1, tgt, g1, l1, s1)
    p.backward(x, g1, dx1, dc1, s1)
    y2, g2, dx2 = (torch.full_like(x, float("nan")) for _ in range(3))
    l2, dc2 = scalar(), coefs()
    p.train_step_mse(x, y2, tgt, g2, l2, dx2, dc2, p.new_saved())
    y3, g3, l3, dc3 = torch.empty_like(x), torch.empty_like(x), scalar(), coefs()
    p.train_step_mse(x, y3, tgt, g3, l3, g3, dc3, p.new_saved())  # dL/dx in g's place
    y4, g4, l4, dc4 = torch.empty_like(x), torch.empty_like(x), scalar(), coefs()
    p.train_step_mse(x, y4, tgt, g4, l4, None, dc4, p.new_saved())
    torch.cuda.synchronize()
    assert p.get_error() == 0
    assert torch.equal(y1, y2) and torch.equal(g1, g2) and torch.equal(dx1, dx2)
    assert torch.equal(y1, y3) and torch.equal(dx1, g3) and torch.equal(y1, y4) and torch.equal(g1, g4)
    for l in (l2, l3, l4):
        assert abs(float(l) - float(l1)) <= 1e-9 * abs(float(l1))
    assert torch.equal(dc2, dc3) and torch.equal(dc2, dc4)
    a, b = dc1.cpu().numpy(), dc2.cpu().numpy()
    for (kind, _), u, v in zip(stages, split(a, stages), split(b, stages)):
        assert np.max(np.abs(u - v)) <= 1e-5 * np.max(np.abs(u)), kind
    lib = oracle.load()
    dx_ref, gref = lib.chain_vjp(xn, g1.cpu().numpy().astype(np.float64), stages)
    assert_close(dx2.cpu().numpy().astype(np.float64), dx_ref, 1e-4, "dL/dx")
    worst = check_coefs(split(b, stages), gref, stages)
    n_two = p.forward_train_mse_launches + p.backward_launches(True, True)
    assert p.train_step_launches(True, True) == (n_two - 1 if spectral else n_two)
    print(f"train step {case}: {d}, coefficient gradients {worst:.2e} of the stage's largest (oracle)")
    p.close()


def test_spectral_8192_points():
    """A chain whose response needs an overlap beyond 3072 samples takes the
    8192-point transforms (the correlation, tap-gradient and decay-check
    kernels at that size): against the oracle, then an update that moves a
    pole to radius 0.9995 is reported as TFX_ERR_DECAY."""
    stages = [("sos", W.random_stable_sos(4, 82, 0.9, 0.99)), ("fir", W.fir_lowpass(1025, 3000.0, W.FS))]
    C, N = 3, 30000
    p = plan(C, N, stages)
    d = p.describe()[0]
    assert d["kind"] == "chain_spectral" and d["M"] == 8192 and 3072 < d["J"] <= 6144, d
    x = W.white_gauss(C, N, 80)
    g = W.white_gauss(C, N, 81)
    y, dx, dc = grads(p, x, g)
    lib = oracle.load()
    assert_close(y, lib.chain(x, stages), 1e-4, "training forward")
    dx_ref, gref = lib.chain_vjp(x, g, stages)
    assert_close(dx, dx_ref, 1e-4, "dL/dx")
    worst = check_coefs(split(dc, stages), gref, stages)
    print(f"8192 points: {d}, worst coefficient error {worst:.2e}")
    rows = np.asarray(stages[0][1]).copy()
    rows[2] = W.biquad_rows([0.0], [-1.0], [[1.0, 0.2, 0.3]], rmin=0.9995, rspan=0.0)[0]
    p.update_sos(torch.from_numpy(rows).cuda())
    torch.cuda.synchronize()
    assert p.get_error() == -8  # TFX_ERR_DECAY
    p.close()


@pytest.mark.parametrize("C,pad", [(1, 0), (3, 13)])
def test_spectral_padded_rows(C, pad):
    """The spectral route with one channel (the correlation's pair has no
    second channel) and with padded rows (row stride N + 13): forward, dL/dx
    and coefficient gradients against the oracle; the padding is not
    written."""
    from paper_2504_08624_gb300 import api, _native
    stages = chain("split_cascades")
    N = 9000
    ld = N + pad
    p = api.Plan(C, N, stages, ld=ld, flags=_native.TFX_PLAN_TRAINABLE)
    assert p.describe()[0]["kind"] == "chain_spectral"
    x = W.white_gauss(C, N, 90)
    g = W.white_gauss(C, N, 91)

    def padded(a, fill):
        buf = torch.full((C * ld,), fill, dtype=torch.float32, device="cuda")
        v = buf.view(C, ld)[:, :N]
        v.copy_(torch.from_numpy(a.astype(np.float32)))
        return buf, v
    _, xd = padded(x, 0.0)
    _, gd = padded(g, 0.0)
    ybuf, y = padded(np.zeros_like(x), -7.0)
    dxbuf, dx = padded(np.zeros_like(x), -7.0)
    dc = torch.empty(p.coef_count, dtype=torch.float64, device="cuda")
    saved = p.new_saved()
    p.forward_train(xd, y, saved)
    p.backward(xd, gd, dx, dc, saved)
    torch.cuda.synchronize()
    assert p.get_error() == 0
    p.close()
    lib = oracle.load()
    assert_close(y.cpu().numpy().astype(np.float64), lib.chain(x, stages), 1e-4, "forward")
    dx_ref, gref = lib.chain_vjp(x, g, stages)
    assert_close(dx.cpu().numpy().astype(np.float64), dx_ref, 1e-4, "dL/dx")
    check_coefs(split(dc.cpu().numpy(), stages), gref, stages)
    if pad:
        assert torch.all(ybuf.view(C, ld)[:, N:] == -7.0) and torch.all(dxbuf.view(C, ld)[:, N:] == -7.0)
