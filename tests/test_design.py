"""Filter designs used to make the workloads' coefficients (inputs, not the
filtering method), checked against their defining properties and scipy."""
import math

import numpy as np
import pytest

from paper_2504_08624_gb300 import workloads as W


def H_sos(rows, f, fs):
    w = 2 * math.pi * np.asarray(f, dtype=np.float64) / fs
    z = np.exp(-1j * w)
    h = np.ones_like(z)
    for b0, b1, b2, a0, a1, a2 in np.asarray(rows).reshape(-1, 6):
        h = h * (b0 + b1 * z + b2 * z * z) / (a0 + a1 * z + a2 * z * z)
    return h


def H_fir(h, f, fs):
    w = 2 * math.pi * np.asarray(f, dtype=np.float64) / fs
    n = np.arange(len(h))
    return np.array([np.sum(h * np.exp(-1j * wi * n)) for wi in np.atleast_1d(w)])


@pytest.mark.parametrize("order", [1, 2, 4, 5, 8])
def test_butterworth_points(order):
    fs, fc = 48000.0, 1000.0
    rows = W.butter_sos(order, fc, fs)
    assert abs(abs(H_sos(rows, 0.0, fs)) - 1.0) < 1e-12
    assert abs(abs(H_sos(rows, fc, fs)) - 1 / math.sqrt(2)) < 1e-12
    assert abs(H_sos(rows, fs / 2, fs)) < 1e-9
    # maximally flat: monotone magnitude
    f = np.linspace(0, fs / 2 * 0.999, 500)
    m = np.abs(H_sos(rows, f, fs))
    assert np.all(np.diff(m) <= 1e-12)
    hp = W.butter_sos(order, fc, fs, "high")
    assert abs(abs(H_sos(hp, fs / 2, fs)) - 1.0) < 1e-12
    assert abs(abs(H_sos(hp, fc, fs)) - 1 / math.sqrt(2)) < 1e-12


@pytest.mark.parametrize("order", [2, 3, 4, 8])
def test_chebyshev1_ripple(order):
    fs, fc, rp = 48000.0, 8000.0, 0.5
    rows = W.cheby1_sos(order, rp, fc, fs)
    g_edge = 10 ** (-rp / 20)
    assert abs(abs(H_sos(rows, fc, fs)) - g_edge) < 1e-10
    f = np.linspace(0, fc, 4000)
    m = np.abs(H_sos(rows, f, fs))
    assert m.max() <= 1 + 1e-9 and m.min() >= g_edge - 1e-9
    assert abs(m.max() - 1.0) < 1e-4
    dc = abs(H_sos(rows, 0.0, fs))
    assert abs(dc - (g_edge if order % 2 == 0 else 1.0)) < 1e-10


def test_peaking_eq():
    fs = 48000.0
    for f0, Q, g in [(100, 0.5, 12.0), (1000, 4.0, -12.0), (9000, 1.3, 3.0)]:
        rows = W.peaking_sos(f0, Q, g, fs)
        assert abs(abs(H_sos(rows, f0, fs)) - 10 ** (g / 20)) < 1e-10
        assert abs(H_sos(rows, 0.0, fs) - 1.0) < 1e-12
        assert abs(H_sos(rows, fs / 2, fs) - 1.0) < 1e-12


def test_fir_designs():
    fs = 48000.0
    h = W.fir_lowpass(1025, 16000.0, fs)
    assert np.max(np.abs(h - h[::-1])) < 1e-16
    assert abs(h.sum() - 1.0) < 1e-12
    hp = W.fir_highpass(101, 100.0, fs)
    assert abs(hp.sum()) < 1e-12
    assert np.max(np.abs(hp - hp[::-1])) < 1e-16
    bp = W.fir_bandpass(16384, 300.0, 3400.0, fs, ("kaiser", 8.0))
    assert np.max(np.abs(bp - bp[::-1])) < 1e-15 * np.max(np.abs(bp))
    assert abs(abs(H_fir(bp, 1850.0, fs)[0]) - 1.0) < 1e-12
    assert abs(H_fir(bp, 20000.0, fs)[0]) < 1e-6


def test_kaiser_i0_series():
    # I0 against its defining integral (1/pi) int_0^pi exp(x cos t) dt
    for x in (0.0, 0.5, 3.0, 8.0, 20.0):
        t = np.linspace(0, math.pi, 200001)
        ref = np.trapezoid(np.exp(x * np.cos(t)), t) / math.pi
        assert abs(W.i0(x) - ref) < 1e-9 * ref


def test_against_scipy():
    sig = pytest.importorskip("scipy.signal")
    fs = 48000.0
    f = np.linspace(10, 23000, 777)
    for order in (2, 4, 8):
        ours = W.butter_sos(order, 1000.0, fs)
        ref = sig.butter(order, 1000.0, fs=fs, output="sos")
        assert np.max(np.abs(H_sos(ours, f, fs) - H_sos(ref, f, fs))) < 1e-9
        ours = W.cheby1_sos(order, 0.5, 8000.0, fs)
        ref = sig.cheby1(order, 0.5, 8000.0, fs=fs, output="sos")
        assert np.max(np.abs(H_sos(ours, f, fs) - H_sos(ref, f, fs))) < 1e-9
    h = W.fir_lowpass(1025, 16000.0, fs)
    ref = sig.firwin(1025, 16000.0, fs=fs, window="hamming")
    assert np.max(np.abs(h - ref)) < 1e-12
    k = W.kaiser(257, 8.0)
    assert np.max(np.abs(k - sig.windows.kaiser(257, 8.0))) < 1e-12


def test_random_sections_are_stable_and_bounded():
    rows = W.random_stable_sos(200, 3)
    for b0, b1, b2, a0, a1, a2 in rows:
        p = np.roots([a0, a1, a2])
        assert np.all(np.abs(p) < 0.9991)
    f = np.linspace(0, 24000, 4096)
    for r in rows[:20]:
        assert np.max(np.abs(H_sos(r, f, 48000.0))) <= 1.0 + 1e-3


def test_signals_are_seeded_and_shaped():
    a = W.pink(2, 48000, 5)
    b = W.pink(2, 48000, 5)
    assert np.array_equal(a, b)
    assert np.allclose(np.sqrt(np.mean(a.astype(np.float64) ** 2, axis=1)), 0.1, rtol=1e-5)
    # 1/f: power in an octave band is roughly constant
    P = np.abs(np.fft.rfft(a[0].astype(np.float64))) ** 2
    lo = P[100:200].sum()
    hi = P[1000:2000].sum()
    assert 0.5 < hi / lo < 2.0
    u = W.white_uniform(3, 1000, 0)
    assert u.dtype == np.float32 and u.min() >= -1 and u.max() <= 1


@pytest.mark.parametrize("kind", ["low", "high"])
@pytest.mark.parametrize("gain", [-9.0, 6.0])
def test_shelving(kind, gain):
    """Shelf gain 10^(G/20) at the shelf end (DC for low, Nyquist for high), 1 at
    the other end, 10^(G/40) at f0."""
    fs, f0 = 48000.0, 2000.0
    rows = W.shelving_sos(kind, f0, gain, fs)
    def H(w):
        z = np.exp(-1j * w)
        r = rows[0]
        return (r[0] + r[1] * z + r[2] * z * z) / (r[3] + r[4] * z + r[5] * z * z)
    g = 10.0 ** (gain / 20.0)
    lo, hi = (g, 1.0) if kind == "low" else (1.0, g)
    assert abs(abs(H(0.0)) - lo) < 1e-12
    assert abs(abs(H(np.pi)) - hi) < 1e-12
    assert abs(abs(H(2 * np.pi * f0 / fs)) - 10.0 ** (gain / 40.0)) < 1e-12


def test_paper_sweep_cells():
    """The paper's timing grid (Sec. 4, Tables 2-3) with its stand-in filters:
    5-600 s x 1-12 channels at 44.1 kHz; the FIR a symmetric 101-tap low-pass
    of unit DC gain, the IIR a 4th-order Butterworth (two sections) at
    1 kHz with |H| = 1/sqrt(2) there; channels and samples of a small cell
    are prefixes of a larger cell's signal."""
    import math
    assert W.PAPER_SWEEP_SECONDS == (5, 60, 180, 300, 600)
    assert W.PAPER_SWEEP_CHANNELS == (1, 2, 4, 8, 12)
    fir = W.paper_sweep("fir", 5, 1)
    assert fir.N == 220500 and fir.C == 1 and fir.tol == 1e-5
    (kind, h), = fir.stages
    h = np.asarray(h)
    assert kind == "fir" and h.size == 101
    assert np.allclose(h, h[::-1], rtol=0, atol=1e-15) and abs(h.sum() - 1.0) < 1e-12
    iir = W.paper_sweep("iir", 600, 12)
    assert iir.N == 26460000 and iir.tol == 1e-4
    (kind, sos), = iir.stages
    sos = np.asarray(sos)
    assert kind == "sos" and sos.shape == (2, 6)
    w = 2 * math.pi * 1000.0 / W.PAPER_SWEEP_FS
    z = np.exp(-1j * np.arange(3) * w)
    H = np.prod([(r[:3] @ z) / (r[3:] @ z) for r in sos])
    assert abs(abs(H) - 2 ** -0.5) < 1e-9
    big = W.paper_sweep("fir", 60, 12).make_signal(3, 1000)
    small = W.paper_sweep("iir", 5, 2).make_signal(2, 500)
    assert np.array_equal(big[:2, :500], small)
    with pytest.raises(ValueError):
        W.paper_sweep("fft", 5, 1)
