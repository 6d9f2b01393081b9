"""tfx_sos_noalloc: the SOS cascade for callers that cannot allocate device
memory (real-time audio callbacks and plug-in hosts, where cudaMalloc's
implicit device synchronisation is not allowed; programs whose device memory
an outside allocator reserves up front).  Its scratch lives in a fixed static
device array.  Checked through the C ABI against tfx_sos, the allocating
entry point, on two calls in a row (the second call finds the first call's
leftovers in the shared array).  Kept in its own file so that it runs last."""
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
    torch.cuda.synchronize()
