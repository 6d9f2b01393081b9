"""The paper's timing grid (Sec. 4, Tables 2 and 3) as the bench runs it:
each filter (the 101-tap FIR, the 4th-order Butterworth) on cells that read
channel and sample prefixes of one wider resident buffer (row stride = the
longest cell's length), against the FP64 oracle per channel.  Tolerance:
1e-5 of each channel's peak for the FIR, 1e-4 for the IIR."""
import numpy as np
import pytest

from paper_2504_08624_gb300 import workloads as W
from tests.gpu_util import assert_close, oracle_chain

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["fir", "iir"])
def test_sweep_cells_from_one_strided_buffer(kind):
    from paper_2504_08624_gb300 import api
    # a 12-channel buffer 7 s long; cells of 1, 2 and 12 channels x 5 s and
    # one ragged length, each a prefix view with the buffer's row stride
    Cmax, Nmax = 12, int(7 * W.PAPER_SWEEP_FS)
    src = W.paper_sweep(kind, 7, Cmax)
    assert src.N == Nmax
    xh = src.make_signal()
    x = torch.from_numpy(xh).cuda()
    for C, N in [(1, int(5 * W.PAPER_SWEEP_FS)), (2, int(5 * W.PAPER_SWEEP_FS)), (12, int(5 * W.PAPER_SWEEP_FS)),
                 (5, 100003)]:
        wl = W.paper_sweep(kind, N / W.PAPER_SWEEP_FS, C)
        assert wl.N == N
        y = torch.full_like(x, -3.0)
        p = api.Plan(C, N, wl.stages, ld=Nmax)
        p.execute(x[:C, :N], y[:C, :N], p.workspace())
        torch.cuda.synchronize()
        assert p.get_error() == 0
        got = y.cpu().numpy()
        assert_close(got[:C, :N], oracle_chain(xh[:C, :N], wl.stages), wl.tol, f"{kind} {C} x {N}")
        # nothing outside the cell is written
        assert np.all(got[:C, N:] == -3.0) and np.all(got[C:] == -3.0)
        p.close()
