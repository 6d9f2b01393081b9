"""Filter design on the GPU in FP64 against the host FP64 designs (which the
design tests pin to |H| at the band edges, ripple and gains), and plan
coefficient updates on the device against freshly built plans and the
oracle.  Error statement: GPU and host designs agree to <= 1e-12 of each
filter's largest coefficient (both FP64; transcendental functions of the
device and the host libm may differ in the last bits)."""
import numpy as np
import pytest

import oracle
from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FS = 48000.0


def host_rows(sp):
    k = sp["kind"]
    if k == "butter_low":
        return W.butter_sos(sp["order"], sp["fc"], FS, "low")
    if k == "butter_high":
        return W.butter_sos(sp["order"], sp["fc"], FS, "high")
    if k == "cheby1_low":
        return W.cheby1_sos(sp["order"], sp["ripple_db"], sp["fc"], FS)
    if k == "peaking":
        return W.peaking_sos(sp["f0"], sp["Q"], sp["gain_db"], FS)
    if k in ("low_shelf", "high_shelf"):
        return W.shelving_sos(k.split("_")[0], sp["f0"], sp["gain_db"], FS, sp.get("slope", 1.0))
    if k == "biquad_polar":
        return W.biquad_rows([sp["rho"]], [sp["phi"]], [sp["b"]])
    raise ValueError(k)


SPECS = ([{"kind": "butter_low", "order": o, "fc": fc} for o in range(1, 11) for fc in (50.0, 1000.0, 15000.0)]
         + [{"kind": "butter_high", "order": o, "fc": fc} for o in (1, 2, 3, 4, 7, 8) for fc in (100.0, 5000.0)]
         + [{"kind": "cheby1_low", "order": o, "ripple_db": rp, "fc": fc} for o in (1, 2, 3, 4, 5, 8)
            for rp in (0.1, 0.5, 3.0) for fc in (800.0, 8000.0)]
         + [{"kind": "peaking", "f0": f0, "Q": q, "gain_db": g} for f0 in (100.0, 3000.0) for q in (0.5, 4.0)
            for g in (-12.0, 9.0)]
         + [{"kind": k, "f0": 2000.0, "gain_db": g, "slope": sl} for k in ("low_shelf", "high_shelf")
            for g in (-6.0, 12.0) for sl in (0.5, 1.0)]
         + [{"kind": "biquad_polar", "rho": r, "phi": p, "b": [0.3, -0.2, 0.1]} for r in (-2.0, 0.0, 3.0)
            for p in (-1.0, 0.5)])


def test_gpu_design_matches_host_designs():
    from paper_2504_08624_gb300 import api
    for sp in SPECS:
        sp.setdefault("fs", FS)
    got = api.design(SPECS)
    worst = 0.0
    for sp, g in zip(SPECS, got):
        ref = host_rows(sp)
        gn = g.cpu().numpy()
        assert gn.shape == ref.shape, sp
        err = np.max(np.abs(gn - ref)) / np.max(np.abs(ref))
        worst = max(worst, err)
        assert err <= 1e-12, (sp, err)
    print(f"worst GPU/host design discrepancy: {worst:.2e} of the largest coefficient")


def test_gpu_design_rejects_invalid_spec():
    from paper_2504_08624_gb300 import api
    with pytest.raises(ValueError):
        api.design([{"kind": "butter_low", "order": 40, "fc": 100.0}])
    with pytest.raises(api.TfxError):
        api.design([{"kind": "butter_low", "order": 4, "fc": 30000.0}])  # above Nyquist: device status


@pytest.mark.parametrize("flags", [0, "trainable", "warp"])
def test_plan_update_sos_on_device(flags):
    from paper_2504_08624_gb300 import api, _native as N
    fl = {0: 0, "trainable": N.TFX_PLAN_TRAINABLE, "warp": N.TFX_PLAN_SCAN_WARP_TILES}[flags]
    rows0 = W.random_stable_sos(5, 3, 0.5, 0.99)
    rows1 = W.random_stable_sos(5, 4, 0.5, 0.99) * np.array([[1.5], [1.0], [0.7], [1.0], [2.0]])  # a0 != 1
    h = W.fir_lowpass(33, 5000.0, FS)
    st0 = [("sos", rows0[:2]), ("fir", h), ("sos", rows0[2:])]
    st1 = [("sos", rows1[:2]), ("fir", h), ("sos", rows1[2:])]
    x = W.white_uniform(2, 40000, 9)
    xd = torch.from_numpy(x).cuda()
    p = api.Plan(2, 40000, st0, flags=fl)
    assert p.sos_rows == 5
    p.update_sos(torch.from_numpy(rows1).cuda())
    y = p.execute(xd).cpu().numpy().astype(np.float64)
    assert p.get_error() == 0
    assert_close(y, oracle.chain(x, st1), 1e-4, "updated plan vs oracle")
    # the same route as the updated plan (an update leaves a composed chain's
    # units running, so the fresh plan keeps its units too; a trainable plan
    # keeps its spectral route and rebuilds the chain's spectrum)
    keep = 0 if flags == "trainable" else N.TFX_PLAN_NO_COMPOSE
    fresh = api.Plan(2, 40000, st1, flags=fl | keep).execute(xd).cpu().numpy().astype(np.float64)
    assert_close(y, fresh, 1e-5, "updated plan vs fresh plan")
    # an unstable row is reported through the status word
    bad = rows1.copy()
    bad[1, 5] = 1.5
    p.update_sos(torch.from_numpy(bad).cuda())
    torch.cuda.synchronize()
    assert p.get_error() == -2
    p.close()


def test_update_then_backward():
    """After a device-side update, the training forward and backward follow the
    new coefficients (the raw rows for the a0 chain rule are updated too)."""
    from paper_2504_08624_gb300 import api, _native as N
    rows0 = W.random_stable_sos(3, 7, 0.5, 0.99)
    rows1 = W.random_stable_sos(3, 8, 0.5, 0.99) * np.array([[2.0], [1.0], [0.5]])
    x = W.white_gauss(2, 5000, 12)
    g = W.white_gauss(2, 5000, 13)
    p = api.Plan(2, 5000, [("sos", rows0)], flags=N.TFX_PLAN_TRAINABLE)
    p.update_sos(torch.from_numpy(rows1).cuda())
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    gd = torch.from_numpy(g.astype(np.float32)).cuda()
    saved = p.new_saved()
    y = torch.empty_like(xd)
    p.forward_train(xd, y, saved)
    dx = torch.empty_like(xd)
    dc = torch.empty(p.coef_count, dtype=torch.float64, device="cuda")
    p.backward(xd, gd, dx, dc, saved)
    torch.cuda.synchronize()
    dx_ref, (gr_ref,) = oracle.load().chain_vjp(x, g, [("sos", rows1)])
    assert_close(dx.cpu().numpy().astype(np.float64), dx_ref, 1e-4, "dx")
    got = dc.cpu().numpy().reshape(3, 6)
    assert np.max(np.abs(got - gr_ref)) <= 1e-4 * np.max(np.abs(gr_ref))
    p.close()
