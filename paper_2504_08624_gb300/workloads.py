"""Seeded synthetic inputs and filter designs for the filter-chain workloads.

This module produces *inputs*: signals and coefficient arrays.  It contains no
filtering arithmetic (no convolution, no difference equation), so both the
CUDA path and the FP64 oracle can take their inputs from it without sharing
any of the method's arithmetic.

Signals (TorchFX Sec. 4 uses seeded white noise at 44.1 kHz):
  * ``white_uniform``  -- U[-1, 1], PCG64 (numpy ``default_rng``).
  * ``white_gauss``    -- N(0, 1), PCG64.
  * ``pink``           -- 1/f-shaped Gaussian: white N(0,1), rfft, bin k>=1
                          scaled by 1/sqrt(k), DC bin zeroed, irfft, each
                          channel normalised to RMS 0.1.

Designs (TorchFX Sec. 3 names Butterworth, Chebyshev, peaking and shelving
filters but gives no formulas; these are the textbook definitions):
  * Butterworth / Chebyshev-I: analog prototype poles, bilinear transform with
    frequency prewarping tan(pi*fc/fs), conjugate poles paired into sections,
    sections ordered by increasing pole radius.  Butterworth fc is the -3 dB
    point; Chebyshev-I fc is the passband edge where the gain first leaves the
    ripple band (-rp dB).
  * Peaking EQ: the RBJ "Audio EQ Cookbook" biquad.
  * Windowed-sinc FIR: symmetric Hamming or Kaiser window over L points;
    low-pass scaled to unit DC gain, high-pass by spectral inversion of a
    unit-DC low-pass (odd L), band-pass as the difference of two low-passes
    scaled to unit gain at the band centre.

Stage lists use the same plain format everywhere:
``[("sos", rows[S x 6] = b0 b1 b2 a0 a1 a2), ("fir", taps[L]), ...]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# signals


def _channel_rng(seed: int, c: int) -> np.random.Generator:
    # one independent PCG64 stream per (seed, channel): any channel subset can
    # be regenerated on its own and matches the full signal
    return np.random.default_rng([int(seed), int(c)])


def white_uniform(C: int, N: int, seed: int, c0: int = 0) -> np.ndarray:
    out = np.empty((C, N), dtype=np.float32)
    for c in range(C):
        v = _channel_rng(seed, c0 + c).random(N, dtype=np.float32)
        out[c] = v * np.float32(2.0) - np.float32(1.0)
    return out


def white_gauss(C: int, N: int, seed: int, c0: int = 0) -> np.ndarray:
    out = np.empty((C, N), dtype=np.float32)
    for c in range(C):
        out[c] = _channel_rng(seed, c0 + c).standard_normal(N, dtype=np.float32)
    return out


def pink(C: int, N: int, seed: int, rms: float = 0.1, c0: int = 0) -> np.ndarray:
    out = np.empty((C, N), dtype=np.float32)
    nb = N // 2 + 1
    scale = np.zeros(nb)
    if nb > 1:
        scale[1:] = 1.0 / np.sqrt(np.arange(1, nb, dtype=np.float64))
    for c in range(C):
        w = _channel_rng(seed, c0 + c).standard_normal(N)
        s = np.fft.irfft(np.fft.rfft(w) * scale, n=N)
        r = math.sqrt(float(np.mean(s * s))) if N else 0.0
        out[c] = (s * (rms / r) if r > 0 else s).astype(np.float32)
    return out


# ----------------------------------------------------------------------------
# IIR designs -> SOS rows (b0 b1 b2 a0 a1 a2), a0 = 1


def _bilinear(p: complex) -> complex:
    # s = (z - 1)/(z + 1)  <=>  z = (1 + s)/(1 - s); prewarping is applied to
    # the analog cutoff, so the prototype is scaled by tan(pi*fc/fs).
    return (1.0 + p) / (1.0 - p)


def _sections_from_poles(zpoles, zero: float, unit_gain_at: float):
    """Build sections from digital poles (one per conjugate pair or real pole).

    Every section gets its zeros at ``zero`` (-1 for low-pass, +1 for
    high-pass) and unit gain at z = ``unit_gain_at`` (1 = DC, -1 = Nyquist).
    Sections are ordered by increasing pole radius."""
    rows = []
    for zp in sorted(zpoles, key=lambda z: abs(z)):
        if abs(zp.imag) > 0.0:
            a = [1.0, -2.0 * zp.real, abs(zp) ** 2]
            b = [1.0, -2.0 * zero, zero * zero]
        else:
            a = [1.0, -zp.real, 0.0]
            b = [1.0, -zero, 0.0]
        u = unit_gain_at
        num = b[0] + b[1] * u + b[2] * u * u
        den = a[0] + a[1] * u + a[2] * u * u
        g = den / num
        rows.append([b[0] * g, b[1] * g, b[2] * g, a[0], a[1], a[2]])
    return np.array(rows, dtype=np.float64)


def _upper_half(poles):
    # one representative per conjugate pair (Im > 0) plus real poles
    out = []
    for p in poles:
        if p.imag > 1e-14:
            out.append(p)
        elif abs(p.imag) <= 1e-14:
            out.append(complex(p.real, 0.0))
    return out


def butter_sos(order: int, fc: float, fs: float, btype: str = "low") -> np.ndarray:
    if order < 1 or not (0.0 < fc < fs / 2):
        raise ValueError("butter_sos: need order >= 1 and 0 < fc < fs/2")
    K = math.tan(math.pi * fc / fs)
    proto = [complex(math.cos(math.pi * (2 * k + order + 1) / (2 * order)),
                     math.sin(math.pi * (2 * k + order + 1) / (2 * order)))
             for k in range(order)]
    if btype == "low":
        analog = [K * q for q in proto]
        zero, ug = -1.0, 1.0
    elif btype == "high":
        analog = [K / q for q in proto]
        zero, ug = 1.0, -1.0
    else:
        raise ValueError("btype must be 'low' or 'high'")
    zp = [_bilinear(p) for p in _upper_half(analog)]
    return _sections_from_poles(zp, zero, ug)


def cheby1_sos(order: int, rp_db: float, fc: float, fs: float) -> np.ndarray:
    """Chebyshev type-I low-pass; fc is the passband edge (gain -rp dB there)."""
    if order < 1 or rp_db <= 0 or not (0.0 < fc < fs / 2):
        raise ValueError("cheby1_sos: bad arguments")
    eps = math.sqrt(10.0 ** (rp_db / 10.0) - 1.0)
    mu = math.asinh(1.0 / eps) / order
    K = math.tan(math.pi * fc / fs)
    proto = []
    for k in range(order):
        th = math.pi * (2 * k + 1) / (2 * order)
        proto.append(complex(-math.sinh(mu) * math.sin(th), math.cosh(mu) * math.cos(th)))
    zp = [_bilinear(K * p) for p in _upper_half(proto)]
    rows = _sections_from_poles(zp, -1.0, 1.0)
    if order % 2 == 0:  # even order: DC sits at the bottom of the ripple band
        rows[0, :3] *= 10.0 ** (-rp_db / 20.0)
    return rows


def peaking_sos(f0: float, Q: float, gain_db: float, fs: float) -> np.ndarray:
    """RBJ peaking-EQ biquad, returned normalised (a0 = 1)."""
    A = 10.0 ** (gain_db / 40.0)
    w0 = 2.0 * math.pi * f0 / fs
    alpha = math.sin(w0) / (2.0 * Q)
    cw = math.cos(w0)
    b = [1.0 + alpha * A, -2.0 * cw, 1.0 - alpha * A]
    a = [1.0 + alpha / A, -2.0 * cw, 1.0 - alpha / A]
    return np.array([[b[0] / a[0], b[1] / a[0], b[2] / a[0], 1.0, a[1] / a[0], a[2] / a[0]]])


def shelving_sos(kind: str, f0: float, gain_db: float, fs: float, slope: float = 1.0) -> np.ndarray:
    """RBJ low/high shelving biquad (shelf slope S), normalised (a0 = 1).  The
    low shelf has gain 10^(G/20) at DC and 1 at Nyquist, the high shelf the
    reverse; both pass 10^(G/40) at f0."""
    A = 10.0 ** (gain_db / 40.0)
    w0 = 2.0 * math.pi * f0 / fs
    cw = math.cos(w0)
    alpha = math.sin(w0) / 2.0 * math.sqrt((A + 1.0 / A) * (1.0 / slope - 1.0) + 2.0)
    q = 2.0 * math.sqrt(A) * alpha
    if kind == "low":
        b = [A * ((A + 1) - (A - 1) * cw + q), 2 * A * ((A - 1) - (A + 1) * cw), A * ((A + 1) - (A - 1) * cw - q)]
        a = [(A + 1) + (A - 1) * cw + q, -2 * ((A - 1) + (A + 1) * cw), (A + 1) + (A - 1) * cw - q]
    elif kind == "high":
        b = [A * ((A + 1) + (A - 1) * cw + q), -2 * A * ((A - 1) + (A + 1) * cw), A * ((A + 1) + (A - 1) * cw - q)]
        a = [(A + 1) - (A - 1) * cw + q, 2 * ((A - 1) - (A + 1) * cw), (A + 1) - (A - 1) * cw - q]
    else:
        raise ValueError("kind must be 'low' or 'high'")
    return np.array([[b[0] / a[0], b[1] / a[0], b[2] / a[0], 1.0, a[1] / a[0], a[2] / a[0]]])


def random_peaking_bank(n: int, fs: float, seed: int) -> np.ndarray:
    """n peaking biquads: f0 log-uniform [100 Hz, 10 kHz], Q log-uniform
    [0.5, 4], gain uniform [-12, 12] dB."""
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        f0 = math.exp(rng.uniform(math.log(100.0), math.log(10000.0)))
        Q = math.exp(rng.uniform(math.log(0.5), math.log(4.0)))
        g = rng.uniform(-12.0, 12.0)
        rows.append(peaking_sos(f0, Q, g, fs)[0])
    return np.array(rows)


def random_stable_sos(n: int, seed: int, rmin: float = 0.3, rmax: float = 0.999,
                      grid: int = 4096) -> np.ndarray:
    """n random stable sections: pole radius U(rmin, rmax), pole angle
    U(0.01 pi, 0.99 pi), zero radius U(0, 1.2), zero angle U(0, pi); each
    section's numerator scaled so that max |H| on a ``grid``-point frequency
    grid is 1."""
    rng = np.random.default_rng(seed)
    w = np.linspace(0.0, math.pi, grid)
    zinv = np.exp(-1j * w)
    rows = []
    for _ in range(n):
        r = rng.uniform(rmin, rmax)
        th = rng.uniform(0.01 * math.pi, 0.99 * math.pi)
        rz = rng.uniform(0.0, 1.2)
        tz = rng.uniform(0.0, math.pi)
        a = np.array([1.0, -2.0 * r * math.cos(th), r * r])
        b = np.array([1.0, -2.0 * rz * math.cos(tz), rz * rz])
        H = (b[0] + b[1] * zinv + b[2] * zinv ** 2) / (a[0] + a[1] * zinv + a[2] * zinv ** 2)
        b = b / float(np.max(np.abs(H)))
        rows.append(np.concatenate([b, a]))
    return np.array(rows)


# ----------------------------------------------------------------------------
# FIR designs


def i0(x: float) -> float:
    """Modified Bessel function of the first kind, order 0, by its power
    series sum_k ((x/2)^k / k!)^2, summed until a term is below 1e-17 of the
    total."""
    s, term, k, hx = 1.0, 1.0, 0, 0.5 * x
    while True:
        k += 1
        term *= (hx / k) ** 2
        s += term
        if term < 1e-17 * s:
            return s


def hamming(L: int) -> np.ndarray:
    if L == 1:
        return np.ones(1)
    n = np.arange(L, dtype=np.float64)
    return 0.54 - 0.46 * np.cos(2.0 * math.pi * n / (L - 1))


def kaiser(L: int, beta: float) -> np.ndarray:
    if L == 1:
        return np.ones(1)
    n = np.arange(L, dtype=np.float64)
    t = 2.0 * n / (L - 1) - 1.0
    den = i0(beta)
    return np.array([i0(beta * math.sqrt(max(0.0, 1.0 - v * v))) / den for v in t])


def _window(L: int, window) -> np.ndarray:
    if window == "hamming":
        return hamming(L)
    if isinstance(window, tuple) and window[0] == "kaiser":
        return kaiser(L, float(window[1]))
    raise ValueError(f"unknown window {window!r}")


def _ideal_lp(L: int, fc: float, fs: float) -> np.ndarray:
    m = np.arange(L, dtype=np.float64) - (L - 1) / 2.0
    f = 2.0 * fc / fs
    return f * np.sinc(f * m)


def fir_lowpass(L: int, fc: float, fs: float, window="hamming") -> np.ndarray:
    h = _ideal_lp(L, fc, fs) * _window(L, window)
    return h / h.sum()


def fir_highpass(L: int, fc: float, fs: float, window="hamming") -> np.ndarray:
    if L % 2 == 0:
        raise ValueError("spectral-inversion high-pass needs an odd tap count")
    h = -fir_lowpass(L, fc, fs, window)
    h[(L - 1) // 2] += 1.0
    return h


def fir_bandpass(L: int, f1: float, f2: float, fs: float, window="hamming") -> np.ndarray:
    if not (0 < f1 < f2 < fs / 2):
        raise ValueError("need 0 < f1 < f2 < fs/2")
    h = (_ideal_lp(L, f2, fs) - _ideal_lp(L, f1, fs)) * _window(L, window)
    w0 = 2.0 * math.pi * 0.5 * (f1 + f2) / fs
    g = abs(np.sum(h * np.exp(-1j * w0 * np.arange(L))))
    return h / g


# ----------------------------------------------------------------------------
# workloads


@dataclass
class Workload:
    name: str
    C: int
    N: int
    stages: list
    tol: float
    signal: str
    seed: int
    meta: dict = field(default_factory=dict)

    def make_signal(self, C: int | None = None, N: int | None = None, c0: int = 0) -> np.ndarray:
        """The seeded input for channels [c0, c0 + C).  White-noise channels are
        prefixes of the full-length channel (N < full length truncates); pink
        noise is shaped over the requested length."""
        C = self.C if C is None else C
        N = self.N if N is None else N
        if self.signal == "uniform":
            return white_uniform(C, N, self.seed, c0)
        if self.signal == "gauss":
            return white_gauss(C, N, self.seed, c0)
        if self.signal == "pink":
            return pink(C, N, self.seed, c0=c0)
        raise ValueError(self.signal)

    @property
    def has_sos(self) -> bool:
        return any(k == "sos" for k, _ in self.stages)

    @property
    def channel_samples(self) -> int:
        return self.C * self.N


FS = 48000.0


def plain_chain() -> Workload:
    """2 ch x 480,000 samples (10 s @ 48 kHz) U[-1,1], seed 0: 4th-order
    Butterworth low-pass 1 kHz (2 sections), then 101-tap Hamming high-pass
    100 Hz."""
    return Workload("plain_chain_2x480000", 2, 480000,
                    [("sos", butter_sos(4, 1000.0, FS)), ("fir", fir_highpass(101, 100.0, FS))],
                    1e-4, "uniform", 0)


def multichannel_fused() -> Workload:
    """64 ch x 2,880,000 samples (60 s @ 48 kHz) pink noise, seed 1:
    8th-order Chebyshev-I low-pass (0.5 dB, 8 kHz; 4 sections), 4 peaking
    biquads (seed 2), then a 1025-tap Hamming low-pass at 16 kHz."""
    return Workload("multichannel_fused_64x2880000", 64, 2880000,
                    [("sos", cheby1_sos(8, 0.5, 8000.0, FS)),
                     ("sos", random_peaking_bank(4, FS, 2)),
                     ("fir", fir_lowpass(1025, 16000.0, FS))],
                    1e-4, "pink", 1)


def long_fir() -> Workload:
    """128 ch x 4,194,304 N(0,1), seed 3: 16384-tap Kaiser(beta=8) band-pass
    300-3400 Hz at 48 kHz."""
    return Workload("long_fir_128x4194304", 128, 4194304,
                    [("fir", fir_bandpass(16384, 300.0, 3400.0, FS, ("kaiser", 8.0)))],
                    1e-5, "gauss", 3)


def biquad_rows(rho, phi, b, rmin: float = 0.5, rspan: float = 0.49) -> np.ndarray:
    """SOS rows of the learnable cascade: pole radius r = rmin + rspan sigmoid(rho)
    (so r stays in (0.5, 0.99)), pole angle theta = pi sigmoid(phi), a = [1,
    -2 r cos theta, r^2]; the numerators b [n x 3] are free."""
    rho, phi, b = np.asarray(rho, float), np.asarray(phi, float), np.asarray(b, float).reshape(-1, 3)
    r = rmin + rspan / (1.0 + np.exp(-rho))
    th = math.pi / (1.0 + np.exp(-phi))
    return np.column_stack([b, np.ones_like(r), -2.0 * r * np.cos(th), r * r])


def differentiable_chain_params(seed: int, n: int = 6, taps: int = 257) -> dict:
    """Parameters of the differentiable chain: n biquads (rho, phi ~ N(0, 1.5),
    numerators from random zeros scaled to max |H| = 1 at the initial poles)
    and a taps-long FIR initialised to a unit impulse plus N(0, 1e-3) noise."""
    rng = np.random.default_rng(seed)
    rho = rng.normal(0.0, 1.5, n)
    phi = rng.normal(0.0, 1.5, n)
    a = biquad_rows(rho, phi, np.ones((n, 3)))[:, 3:]
    w = np.linspace(0.0, math.pi, 4096)
    zinv = np.exp(-1j * w)
    b = np.empty((n, 3))
    for i in range(n):
        rz, tz = rng.uniform(0.0, 1.2), rng.uniform(0.0, math.pi)
        bi = np.array([1.0, -2.0 * rz * math.cos(tz), rz * rz])
        H = (bi[0] + bi[1] * zinv + bi[2] * zinv ** 2) / (a[i, 0] + a[i, 1] * zinv + a[i, 2] * zinv ** 2)
        b[i] = bi / float(np.max(np.abs(H)))
    h = rng.normal(0.0, 1e-3, taps)
    h[0] += 1.0
    return {"rho": rho, "phi": phi, "b": b, "h": h}


def differentiable_chain_forward() -> Workload:
    """256 x 65,536 N(0,1), seed 4: the learnable chain at its initial
    parameters (seed 41): 6 biquads with poles parameterised by radius in
    (0.5, 0.99) and angle, free numerators, then a 257-tap FIR (unit impulse
    plus N(0, 1e-3) noise).  Trained with the MSE to ``differentiable_chain_target``."""
    p = differentiable_chain_params(41)
    return Workload("differentiable_chain_256x65536", 256, 65536,
                    [("sos", biquad_rows(p["rho"], p["phi"], p["b"])), ("fir", p["h"])],
                    1e-4, "gauss", 4, meta={"params": p})


def differentiable_chain_target() -> list:
    """The target chain: the same architecture with parameters from seed 141."""
    p = differentiable_chain_params(141)
    return [("sos", biquad_rows(p["rho"], p["phi"], p["b"])), ("fir", p["h"])]


def table4_chain() -> Workload:
    """8 ch x 120 s @ 44.1 kHz N(0,1): two 4th-order Butterworth low-passes
    (1 kHz, 5 kHz) and two 4th-order Chebyshev-I (0.5 dB; 2 kHz, 8 kHz)."""
    fs = 44100.0
    return Workload("table4_chain_8x5292000", 8, int(120 * fs),
                    [("sos", butter_sos(4, 1000.0, fs)), ("sos", butter_sos(4, 5000.0, fs)),
                     ("sos", cheby1_sos(4, 0.5, 2000.0, fs)), ("sos", cheby1_sos(4, 0.5, 8000.0, fs))],
                    1e-4, "gauss", 6)


def random_chain(seed: int, max_sections: int = 8, min_taps: int = 33, max_taps: int = 2049):
    """One random chain: U{1..max_sections} random stable sections (radius
    0.3-0.999) then an FIR with round(log-uniform[min_taps, max_taps]) taps
    forced odd, Hamming low-pass with fc ~ U(0.05, 0.45) fs."""
    rng = np.random.default_rng(seed)
    S = int(rng.integers(1, max_sections + 1))
    L = int(round(math.exp(rng.uniform(math.log(min_taps), math.log(max_taps)))))
    L |= 1
    fc = rng.uniform(0.05, 0.45) * FS
    return [("sos", random_stable_sos(S, seed + 7919)), ("fir", fir_lowpass(L, fc, FS))]


@dataclass
class Clip:
    """One clip of the batched workload: C channels x N samples of U[-1, 1]
    noise (seed) through its own chain."""
    C: int
    N: int
    stages: list
    seed: int

    def make_signal(self) -> np.ndarray:
        return white_uniform(self.C, self.N, self.seed)


def batched_clips(n: int = 1000, seed: int = 5) -> list:
    """The many-clip workload (c13): lengths round(48000 exp(U(ln 0.5, ln 30)))
    samples, channels from {1, 2, 6, 8, 16}, each clip with its own chain of
    1-8 random stable sections (pole radius <= 0.999) and a Hamming low-pass
    FIR of log-uniform 33-2049 taps (odd, fc ~ U(0.05, 0.45) fs)."""
    rng = np.random.default_rng(seed)
    clips = []
    for i in range(n):
        N = int(round(FS * math.exp(rng.uniform(math.log(0.5), math.log(30.0)))))
        C = int(rng.choice([1, 2, 6, 8, 16]))
        clips.append(Clip(C, N, random_chain(seed * 100003 + i), seed * 1000003 + i))
    return clips


# The paper's timing grid (Sec. 4, Tables 2 and 3): signal durations in
# seconds and channel counts, 44.1 kHz Gaussian noise, one filter at a time.
PAPER_SWEEP_SECONDS = (5, 60, 180, 300, 600)
PAPER_SWEEP_CHANNELS = (1, 2, 4, 8, 12)
PAPER_SWEEP_FS = 44100.0


def paper_sweep(kind: str, seconds: float, C: int) -> Workload:
    """One cell of the paper's timing grid: C channels x `seconds` of N(0, 1)
    noise at 44.1 kHz through ONE filter, kind "fir" (a 101-tap Hamming
    low-pass at 1 kHz) or "iir" (a 4th-order Butterworth low-pass at 1 kHz,
    two sections).  The paper states neither the FIR's taps nor the IIR's
    order: these are stand-ins.  Channels and samples are prefixes of the
    largest cell's signal (seed 7), so one buffer serves every cell."""
    fs = PAPER_SWEEP_FS
    N = int(round(seconds * fs))
    if kind == "fir":
        stages, tol = [("fir", fir_lowpass(101, 1000.0, fs))], 1e-5
    elif kind == "iir":
        stages, tol = [("sos", butter_sos(4, 1000.0, fs))], 1e-4
    else:
        raise ValueError(f"paper_sweep: kind must be 'fir' or 'iir', not {kind!r}")
    return Workload(f"paper_sweep_{kind}_{C}x{N}", C, N, stages, tol, "gauss", 7,
                    meta={"kind": kind, "seconds": seconds})


WORKLOADS = {
    "plain_chain": plain_chain,
    "multichannel_fused": multichannel_fused,
    "long_fir": long_fir,
    "differentiable_chain": differentiable_chain_forward,
    "table4_chain": table4_chain,
}
