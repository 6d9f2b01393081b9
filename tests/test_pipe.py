"""The pipe operator (Sec. 3): signal | filter | filter, lazy sample-rate
binding, nn.Sequential piping, and one fused library call per piped chain."""
import numpy as np
import pytest

from paper_2504_08624_gb300 import workloads as W

torch = pytest.importorskip("torch")
from paper_2504_08624_gb300 import pipe as P  # noqa: E402


def test_filter_composition_binds_rate_late():
    chain = P.Butterworth(4, 1000.0) | P.WindowedSinc(101, 100.0, "high")
    st = chain.stages(48000.0)
    ref = W.plain_chain().stages
    assert [k for k, _ in st] == [k for k, _ in ref]
    for (_, a), (_, b) in zip(st, ref):
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))
    # the same filter objects at another rate design other coefficients
    st44 = chain.stages(44100.0)
    assert not np.allclose(st44[0][1], st[0][1])


def test_pipe_records_without_running():
    x = torch.zeros(2, 1000)  # host tensor: nothing runs until .y is read
    seq = torch.nn.Sequential(P.HiShelving(1000.0), P.LoShelving(2000.0))
    s = P.Signal(x, 48000.0) | seq | P.Peaking(3000.0, 2.0, 6.0)
    assert s.pending_stages == 3
    s2 = s | (P.Butterworth(2, 500.0) | P.FIR([1.0, 0.5]))
    assert s2.pending_stages == 5 and s.pending_stages == 3


def test_filter_without_rate_refuses_forward():
    with pytest.raises(ValueError):
        P.Butterworth(2, 500.0)(torch.zeros(1, 10))


def test_pipe_rejects_non_filters():
    with pytest.raises(TypeError):
        P.Signal(torch.zeros(1, 10), 48000.0) | 3


@pytest.mark.gpu
def test_pipe_matches_oracle_and_runs_fused():
    import oracle
    from tests.gpu_util import assert_close
    fs = 48000.0
    x = W.white_uniform(3, 20000, 7)
    sig = P.Signal(torch.from_numpy(x).cuda(), fs)
    seq = torch.nn.Sequential(P.HiShelving(1000.0), P.LoShelving(2000.0, gain_db=-4.0))
    out = sig | seq | P.Chebyshev1(4, 0.5, 8000.0) | P.WindowedSinc(257, 6000.0)
    assert out.pending_stages == 4
    y = out.y.cpu().numpy().astype(np.float64)
    assert out.pending_stages == 0
    stages = (P.Chain([seq]) | P.Chebyshev1(4, 0.5, 8000.0) | P.WindowedSinc(257, 6000.0)).stages(fs)
    assert_close(y, oracle.chain(x, stages), 1e-4, "pipe")
    # a filter module applied directly at a bound rate
    f = P.Butterworth(4, 1000.0, fs=fs)
    y2 = f(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    assert_close(y2, oracle.chain(x, f.stages(fs)), 1e-4, "module forward")
