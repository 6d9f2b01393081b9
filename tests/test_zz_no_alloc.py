"""tfx_sos_noalloc: the SOS cascade for callers that cannot allocate device
memory (real-time audio callbacks and plug-in hosts, where cudaMalloc's
implicit device synchronisation is not allowed; programs whose device memory
an outside allocator reserves up front).  Its scratch lives in a fixed static
device array.  Checked through the C ABI against tfx_sos, the allocating
entry point, on two calls in a row (the second call finds the first call's
leftovers in the shared array), and against the FP64 oracle directly, in
place and with padded rows.  Kept in its own file so that it runs last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.gpu
def test_noalloc_matches_tfx_sos_on_two_calls():
    from paper_2504_08624_gb300 import _native as N, workloads as W
    from tests.gpu_util import assert_close
    lib = N.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sos = np.ascontiguousarray(np.concatenate([W.cheby1_sos(8, 0.5, 8000.0, 48000.0),
                                               W.random_peaking_bank(4, 48000.0, 2)]))
    sp = sos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for call, (C, Ns) in enumerate([(3, 3 * 8192 + 123), (5, 2 * 8192 + 7)]):
        x = torch.from_numpy(W.white_uniform(C, Ns, 90 + call)).cuda()
        y_ref = torch.empty_like(x)
        y_na = torch.full_like(x, float("nan"))
        assert lib.tfx_sos(_ptr(x), _ptr(y_ref), C, Ns, Ns, sp, sos.shape[0], stream) == 0
        assert lib.tfx_sos_noalloc(_ptr(x), _ptr(y_na), C, Ns, Ns, sp, sos.shape[0], stream) == 0
        torch.cuda.synchronize()
        assert_close(y_na.cpu().numpy(), y_ref.cpu().numpy().astype(np.float64), 1e-4,
                     f"noalloc call {call}")


@pytest.mark.gpu
def test_noalloc_matches_oracle_inplace_and_padded():
    """Against the FP64 oracle: an in-place call (x == y) and a call on rows
    padded to a longer stride (ld > N), each over several 8192-sample tiles."""
    import oracle
    from paper_2504_08624_gb300 import _native as N, workloads as W
    from tests.gpu_util import assert_close
    lib = N.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sos = np.ascontiguousarray(np.concatenate([W.butter_sos(4, 1000.0, 48000.0),
                                               W.random_stable_sos(3, 77, 0.5, 0.999)]))
    sp = sos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    C, Ns = 3, 5 * 8192 + 333
    x = W.white_uniform(C, Ns, 93)
    ref = oracle.chain(x, [("sos", sos)])
    # in place
    xt = torch.from_numpy(x).cuda()
    assert lib.tfx_sos_noalloc(_ptr(xt), _ptr(xt), C, Ns, Ns, sp, sos.shape[0], stream) == 0
    torch.cuda.synchronize()
    assert_close(xt.cpu().numpy(), ref, 1e-4, "noalloc in place")
    # padded rows: ld = Ns + 77, the padding must stay untouched
    ld = Ns + 77
    xp = torch.full((C, ld), 7.0, dtype=torch.float32, device="cuda")
    xp[:, :Ns] = torch.from_numpy(x).cuda()
    yp = torch.full((C, ld), -3.0, dtype=torch.float32, device="cuda")
    assert lib.tfx_sos_noalloc(_ptr(xp), _ptr(yp), C, Ns, ld, sp, sos.shape[0], stream) == 0
    torch.cuda.synchronize()
    assert_close(yp[:, :Ns].cpu().numpy(), ref, 1e-4, "noalloc padded rows")
    assert torch.all(yp[:, Ns:] == -3.0)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2504_08624_gb300 import _native as N, workloads as W
    lib = N.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    sos9 = np.ascontiguousarray(np.tile(W.butter_sos(2, 1000.0, 48000.0)[:1], (9, 1)))
    sp9 = sos9.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.tfx_sos_noalloc(_ptr(x), _ptr(x), 1, 16, 16, sp9, 9, stream) == -6   # > 8 sections
    sos1 = np.ascontiguousarray(W.butter_sos(2, 1000.0, 48000.0))
    sp1 = sos1.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    # 40000 channels x 2 tiles > 32768 tiles: rejected before anything is enqueued
    assert lib.tfx_sos_noalloc(_ptr(x), _ptr(x), 40000, 8193, 8193, sp1, 1, stream) == -6
    # a pole of radius 0.9995 (beyond 0.999, where the plans switch to FP64
    # carries): this entry point keeps FP32 carries and refuses it
    r, th = 0.9995, 0.05
    hi = np.ascontiguousarray([[1.0, 0.0, 0.0, 1.0, -2 * r * np.cos(th), r * r]])
    sph = hi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.tfx_sos_noalloc(_ptr(x), _ptr(x), 1, 16, 16, sph, 1, stream) == -6
    torch.cuda.synchronize()
