"""The FP64 oracle against closed forms, brute force and exact identities.

Nothing here compares the oracle with itself: each pin (see ``pins.py``) is a
value fixed by the mathematics of the difference equation / convolution
(TorchFX Sec. 3, lfilter semantics; Sec. 4 workloads), or an independent
library routine (scipy.signal) where available.
"""
import numpy as np
import pytest

import oracle
from tests import pins


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(lib, pin):
    pin(lib, np.random.default_rng(1234))


def test_edge_cases(lib):
    # empty signals
    assert lib.sos(np.zeros((0, 5)), [1, 0, 0, 1, 0, 0]).shape == (0, 5)
    assert lib.fir(np.zeros((3, 0)), [1.0]).shape == (3, 0)
    # identity section and single-tap gain
    x = np.random.default_rng(0).standard_normal((2, 50))
    assert np.array_equal(lib.sos(x, [1, 0, 0, 1, 0, 0]), x)
    assert np.array_equal(lib.fir(x, [2.0]), 2.0 * x)
    # taps longer than the signal
    h = np.arange(1.0, 101.0)
    y = lib.fir(np.ones(10), h)
    assert np.array_equal(y, np.cumsum(h[:10]))
    # zero sections is the identity; a0 = 0 is rejected
    assert np.array_equal(lib.chain(x, [("sos", np.zeros((0, 6)))]), x)
    with pytest.raises(ValueError):
        lib.sos(x, [1, 0, 0, 0, 0, 0])
    with pytest.raises(ValueError):
        lib.fir(x, [])


def test_scipy_cross_check(lib):
    """Independent library route: scipy.signal.sosfilt / lfilter in float64."""
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(7)
    from paper_2504_08624_gb300 import workloads as W
    sos = np.concatenate([W.cheby1_sos(8, 0.5, 8000, 48000), W.random_peaking_bank(4, 48000, 2)])
    x = rng.standard_normal((3, 20000))
    got = lib.sos(x, sos)
    want = sig.sosfilt(sos, x, axis=-1)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    h = W.fir_lowpass(1025, 16000, 48000)
    got = lib.fir(x, h)
    want = sig.lfilter(h, [1.0], x, axis=-1)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))
    # non-normalised rows (a0 != 1) against lfilter's own normalisation
    row = np.array([0.4, 0.2, 0.1, 2.0, -1.2, 0.5])
    got = lib.sos(x, row)
    want = sig.lfilter(row[:3], row[3:], x, axis=-1)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_chain_matches_stagewise_definition(lib):
    """The chain is defined as list-order composition (TorchFX Sec. 3, pipe
    operator); with scipy as the stage implementation."""
    sig = pytest.importorskip("scipy.signal")
    from paper_2504_08624_gb300 import workloads as W
    wl = W.plain_chain()
    x = wl.make_signal(2, 30000)
    want = x.astype(np.float64)
    for kind, coef in wl.stages:
        if kind == "sos":
            want = sig.sosfilt(coef, want, axis=-1)
        else:
            want = sig.lfilter(coef, [1.0], want, axis=-1)
    got = lib.chain(x, wl.stages)
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_property_random_sections(lib):
    hyp = pytest.importorskip("hypothesis")
    from hypothesis import given, settings, strategies as st

    @settings(max_examples=60, deadline=None)
    @given(r=st.floats(0.05, 0.999), th=st.floats(0.01, 3.13),
           b=st.lists(st.floats(-2, 2), min_size=3, max_size=3),
           a0=st.floats(0.25, 4.0), N=st.integers(1, 300))
    def check(r, th, b, a0, N):
        row = np.array([b[0], b[1], b[2], a0, -2 * r * np.cos(th) * a0, r * r * a0])
        x = np.zeros(N)
        x[0] = 1.0
        got = lib.sos(x, row)
        want = pins.biquad_impulse_closed_form(row, N)
        scale = max(1e-12, float(np.max(np.abs(want))))
        assert np.max(np.abs(got - want)) <= 1e-9 * scale

    check()


def test_threads_reported(lib):
    assert lib.num_threads() >= 1
