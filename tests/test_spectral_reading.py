"""Reading R15 of the design (training by the composite spectrum): the chain
is linear and time-invariant (TorchFX Sec. 3: the pipe composes the
stages), so for L = sum g y
    dL/dtheta = sum_(j >= 0) (dh/dtheta)[j] r[j],  r[j] = sum_c sum_n g[c][n] x[c][n - j],
and dL/dx is the chain applied to g in reverse time.  The plan's spectral
route evaluates the derivative spectra in closed form at M bins
(dH/db_k = z^k F prod_(j != s) H_j / A_s, dH/da_k = -z^k H / A_s,
dH/dh_k = z^k prod_s H_s, z = e^(-i w), sections a0-normalised), takes r at
lags 0..J from block cross-spectra (B = M - J gradient samples after J
zeros against the window of J + B input samples), and needs the derivative
responses to have decayed within J.

Here that reading is written out in code of the test's own (numpy FP64,
one channel per transform, the a0 chain rule by hand) and checked against
the FP64 oracle's forward-mode vector-Jacobian product: it matches at an
overlap the responses have outlived, and misses by far more at an overlap
they have not (so the check is sensitive).  No GPU."""
import numpy as np

import oracle
from paper_2504_08624_gb300 import workloads as W


def _spectral_vjp(x, g, rows, taps, M, J):
    """(dL/dx, dL/d rows [S x 6], dL/d taps) by the reading, FP64."""
    C, N = x.shape
    B = M - J
    k = np.arange(M)
    z = np.exp(-2j * np.pi * k / M)
    a0 = rows[:, 3:4]
    nr = rows / a0  # b0 b1 b2 1 a1 a2
    Bs = nr[:, 0:1] + nr[:, 1:2] * z + nr[:, 2:3] * z ** 2
    As = 1.0 + nr[:, 4:5] * z + nr[:, 5:6] * z ** 2
    Hs = Bs / As
    F = np.fft.fft(taps, M)
    Cs = np.prod(Hs, axis=0)
    H = F * Cs
    # cross-spectrum of the gradient blocks (after J zeros) and input windows
    S = np.zeros(M, complex)
    for c in range(C):
        for n0 in range(0, N, B):
            win = np.zeros(M)
            lo = n0 - J
            seg = x[c, max(lo, 0):min(n0 + B, N)]
            win[max(lo, 0) - lo:max(lo, 0) - lo + seg.size] = seg
            gb = np.zeros(M)
            gs = g[c, n0:min(n0 + B, N)]
            gb[J:J + gs.size] = gs
            S += np.fft.fft(gb) * np.conj(np.fft.fft(win))
    inner = lambda d: float(np.real(np.sum(np.conj(d) * S)) / M)
    grows = np.zeros_like(rows)
    for s in range(rows.shape[0]):
        others = F * np.prod(np.delete(Hs, s, axis=0), axis=0)
        G = [inner(z ** q * others / As[s]) for q in range(3)]       # d/d b_q (normalised)
        G += [inner(-(z ** q) * H / As[s]) for q in (1, 2)]           # d/d a_q (normalised)
        inv = 1.0 / rows[s, 3]
        grows[s, [0, 1, 2, 4, 5]] = np.array(G) * inv
        grows[s, 3] = -(rows[s, 0] * G[0] + rows[s, 1] * G[1] + rows[s, 2] * G[2]
                        + rows[s, 4] * G[3] + rows[s, 5] * G[4]) * inv * inv
    gtaps = np.real(np.fft.ifft(np.conj(Cs) * S))[:taps.size]
    # dL/dx: the chain (spectrum H, overlap J) over the gradient in reverse time
    dx = np.zeros_like(x)
    for c in range(C):
        gr = g[c, ::-1]
        out = np.zeros(N)
        for n0 in range(0, N, B):
            win = np.zeros(M)
            lo = n0 - J
            seg = gr[max(lo, 0):min(n0 + B, N)]
            win[max(lo, 0) - lo:max(lo, 0) - lo + seg.size] = seg
            yb = np.real(np.fft.ifft(np.fft.fft(win) * H))
            m = min(B, N - n0)
            out[n0:n0 + m] = yb[J:J + m]
        dx[c] = out[::-1]
    return dx, grows, gtaps


def _case():
    rows = W.random_stable_sos(3, 91, 0.5, 0.9) * np.array([[1.5], [1.0], [0.8]])
    taps = np.random.default_rng(92).normal(0.0, 0.2, 33)
    x = W.white_gauss(2, 5000, 93).astype(np.float64)
    g = W.white_gauss(2, 5000, 94).astype(np.float64)
    return rows, taps, x, g


def test_spectral_vjp_matches_the_oracle():
    rows, taps, x, g = _case()
    stages = [("sos", rows), ("fir", taps)]
    dx_ref, (gr_ref, gt_ref) = oracle.load().chain_vjp(x, g, stages)
    dx, gr, gt = _spectral_vjp(x, g, rows, taps, M=1024, J=400)
    assert np.max(np.abs(gr - gr_ref)) <= 1e-9 * np.max(np.abs(gr_ref))
    assert np.max(np.abs(gt - gt_ref)) <= 1e-9 * np.max(np.abs(gt_ref))
    assert np.max(np.abs(dx - dx_ref)) <= 1e-9 * np.max(np.abs(dx_ref))


def test_short_overlap_is_detected_by_the_check():
    """An overlap the derivative responses have not outlived misses by far
    more than the tolerance (the decay requirement is not vacuous)."""
    rows, taps, x, g = _case()
    stages = [("sos", rows), ("fir", taps)]
    _, (gr_ref, gt_ref) = oracle.load().chain_vjp(x, g, stages, want_dx=False)
    _, gr, gt = _spectral_vjp(x, g, rows, taps, M=1024, J=40)
    assert np.max(np.abs(gr - gr_ref)) > 1e-3 * np.max(np.abs(gr_ref))
