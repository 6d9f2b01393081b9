"""Closed-form and brute-force pins for the FP64 oracle.

Every function takes an oracle library handle (``oracle.load(...)``) and raises
AssertionError when the oracle disagrees with something fixed by mathematics
rather than by the oracle itself: closed-form impulse responses, steady-state
gains read off the transfer function, explicit matrix (Toeplitz / banded
triangular) formulations, and exact identities.  ``tests/test_oracle.py`` runs
them against the oracle; ``tests/test_oracle_plants.py`` runs them against
builds with one planted mistake each and checks that some pin fails.
"""
import math

import numpy as np


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(1e-300, float(np.max(np.abs(b)))))


def biquad_impulse_closed_form(row, N):
    """Impulse response of one section from its poles (TorchFX Sec. 3: the
    lfilter difference equation; here solved in closed form).

    With alpha = a/a0 and poles p1, p2 of z^2 + alpha1 z + alpha2, the
    all-pole part has g[n] = (p1^(n+1) - p2^(n+1)) / (p1 - p2) (distinct poles;
    r^n sin((n+1) theta)/sin(theta) for a conjugate pair, (n+1) p^n for a
    double pole) and h[n] = (b0 g[n] + b1 g[n-1] + b2 g[n-2]) / a0."""
    b0, b1, b2, a0, a1, a2 = [float(v) for v in row]
    al1, al2 = a1 / a0, a2 / a0
    n = np.arange(N, dtype=np.float64)
    disc = al1 * al1 - 4.0 * al2
    tiny = 1e-12 * max(1.0, al1 * al1)
    if disc < -tiny:
        r = math.sqrt(al2)
        th = math.acos(max(-1.0, min(1.0, -al1 / (2.0 * r))))
        g = r ** n * np.sin((n + 1) * th) / math.sin(th)
    elif disc > tiny:
        sq = math.sqrt(disc)
        p1, p2 = (-al1 + sq) / 2.0, (-al1 - sq) / 2.0
        g = (p1 ** (n + 1) - p2 ** (n + 1)) / (p1 - p2)
    else:
        p = -al1 / 2.0
        g = (n + 1) * p ** n
    h = b0 * g
    h[1:] += b1 * g[:-1]
    h[2:] += b2 * g[:-2]
    return h / a0


def freq_response(row, w):
    b0, b1, b2, a0, a1, a2 = [float(v) for v in row]
    z = np.exp(-1j * np.asarray(w, dtype=np.float64))
    return (b0 + b1 * z + b2 * z * z) / (a0 + a1 * z + a2 * z * z)


# --- FIR pins ----------------------------------------------------------------


def pin_fir_impulse(lib, rng):
    """A unit impulse returns the taps exactly (then zeros)."""
    L = 37
    h = rng.standard_normal(L)
    for N in (1, 20, 37, 80):
        x = np.zeros(N)
        x[0] = 1.0
        y = lib.fir(x, h)
        want = np.zeros(N)
        m = min(N, L)
        want[:m] = h[:m]
        assert np.array_equal(y, want), f"FIR impulse mismatch at N={N}"


def pin_fir_toeplitz(lib, rng):
    """Against the explicit N x N lower-triangular Toeplitz matrix product."""
    for N, L in ((1, 1), (5, 9), (64, 17), (200, 33), (256, 256)):
        h = rng.standard_normal(L)
        x = rng.standard_normal((3, N))
        T = np.zeros((N, N))
        for i in range(N):
            for k in range(min(L, i + 1)):
                T[i, i - k] = h[k]
        want = x @ T.T
        got = lib.fir(x, h)
        assert _rel(got, want) < 1e-13, f"FIR Toeplitz mismatch N={N} L={L}"


def pin_fir_at_sampled(lib, rng):
    """The FIR at chosen output positions: a unit impulse at position p gives
    h[n - p] at every sampled n (zero before p and beyond p + L - 1), and a
    random signal gives the rows of the explicit Toeplitz matrix product at
    the sampled positions, including the first outputs (fewer than L terms)."""
    L, N, p = 29, 300, 41
    h = rng.standard_normal(L)
    x = np.zeros(N)
    x[p] = 1.0
    idx = np.array([0, p - 1, p, p + 5, p + L - 1, p + L, N - 1])
    want = np.array([h[n - p] if 0 <= n - p < L else 0.0 for n in idx])
    assert np.array_equal(lib.fir_at(x, h, idx), want), "sampled FIR impulse mismatch"
    x = rng.standard_normal(N)
    T = np.zeros((N, N))
    for i in range(N):
        for k in range(min(L, i + 1)):
            T[i, i - k] = h[k]
    idx = np.array([0, 1, L - 2, L - 1, L, 150, N - 1])
    assert _rel(lib.fir_at(x, h, idx), (T @ x)[idx]) < 1e-13, "sampled FIR Toeplitz mismatch"


def pin_fir_dc_nyquist(lib, rng):
    """Constant input gives sum(h) once the delay line is full; (-1)^n gives
    (-1)^n sum_k (-1)^k h[k]."""
    L = 41
    h = rng.standard_normal(L)
    N = 200
    n = np.arange(N)
    y = lib.fir(np.ones(N), h)
    assert abs(y[L - 1:] - h.sum()).max() < 1e-12 * max(1.0, abs(h).sum())
    alt = (-1.0) ** n
    y = lib.fir(alt, h)
    g = np.sum(h * (-1.0) ** np.arange(L))
    assert abs(y[L - 1:] - alt[L - 1:] * g).max() < 1e-12 * max(1.0, abs(h).sum())


# --- SOS pins ----------------------------------------------------------------


def _rows_for_pins():
    """Sections covering conjugate, distinct-real and repeated-real poles,
    a0 != 1, and radii up to 0.999."""
    rows = []
    for r, th in ((0.5, 0.3), (0.9, 1.1), (0.99, 0.05), (0.999, 2.5)):
        rows.append([0.7, -0.2, 0.4, 1.0, -2 * r * math.cos(th), r * r])
    rows.append([1.0, 0.5, 0.25, 1.0, -(0.8 + 0.3), 0.8 * 0.3])     # distinct real
    rows.append([0.3, 0.6, 0.3, 1.0, -2 * 0.7, 0.49])              # double pole 0.7
    rows.append([2.0, 1.0, -0.5, 2.5, -2.5 * 1.2, 2.5 * 0.6])      # a0 = 2.5
    rows.append([0.5, 0.0, 0.0, 1.0, -0.95, 0.0])                  # first order
    return [np.array(r, dtype=np.float64) for r in rows]


def pin_sos_impulse_closed_form(lib, rng):
    for row in _rows_for_pins():
        N = 600
        x = np.zeros(N)
        x[0] = 1.0
        got = lib.sos(x, row)
        want = biquad_impulse_closed_form(row, N)
        assert _rel(got, want) < 1e-10, f"SOS impulse mismatch for {row}"


def pin_sos_steady_state(lib, rng):
    """DC, Nyquist and sinusoidal steady state equal H(e^jw) read off the
    coefficients once the transient has decayed."""
    for row in _rows_for_pins():
        al2 = row[5] / row[3]
        al1 = row[4] / row[3]
        rad = max(abs(np.roots([1.0, al1, al2]))) if al2 != 0 else abs(al1)
        n_tr = int(math.ceil(math.log(1e-15) / math.log(max(rad, 1e-3)))) + 50
        N = n_tr + 64
        n = np.arange(N)
        for w in (0.0, math.pi, 0.37, 1.9):
            x = np.cos(w * n)
            H = freq_response(row, w)
            want = abs(H) * np.cos(w * n + np.angle(H))
            got = lib.sos(x, row)
            scale = max(1.0, abs(H))
            assert np.max(np.abs(got[n_tr:] - want[n_tr:])) < 1e-9 * scale, \
                f"steady state mismatch row={row} w={w}"


def pin_sos_banded_solve(lib, rng):
    """y = A^-1 B x with A, B the banded lower-triangular matrices of the
    difference equation (dense triangular solve)."""
    from numpy.linalg import solve
    for row in _rows_for_pins():
        N = 120
        b0, b1, b2, a0, a1, a2 = row
        A = np.zeros((N, N))
        B = np.zeros((N, N))
        for i in range(N):
            A[i, i], B[i, i] = a0, b0
            if i >= 1:
                A[i, i - 1], B[i, i - 1] = a1, b1
            if i >= 2:
                A[i, i - 2], B[i, i - 2] = a2, b2
        x = rng.standard_normal((2, N))
        want = solve(A, B @ x.T).T
        got = lib.sos(x, row)
        assert _rel(got, want) < 1e-9, f"banded solve mismatch row={row}"


def pin_sos_scale_invariance(lib, rng):
    """Scaling all six coefficients of a row leaves the output unchanged."""
    x = rng.standard_normal((2, 300))
    for row in _rows_for_pins():
        y1 = lib.sos(x, row)
        y2 = lib.sos(x, row * 3.7)
        assert _rel(y2, y1) < 1e-12


def pin_cascade_closed_form(lib, rng):
    """Impulse response of a cascade = convolution of the sections' closed-form
    impulse responses; cascade order does not matter (up to rounding)."""
    rows = _rows_for_pins()[:4]
    N = 500
    want = np.zeros(N)
    want[0] = 1.0
    for r in rows:
        want = np.convolve(want, biquad_impulse_closed_form(r, N))[:N]
    x = np.zeros(N)
    x[0] = 1.0
    got = lib.sos(x, np.stack(rows))
    assert _rel(got, want) < 1e-9
    xs = rng.standard_normal((2, 700))
    y_fwd = lib.sos(xs, np.stack(rows))
    y_rev = lib.sos(xs, np.stack(rows[::-1]))
    assert _rel(y_rev, y_fwd) < 1e-10


def pin_chain_closed_form(lib, rng):
    """Chain [SOS cascade, FIR]: impulse response = closed-form cascade
    response convolved with the taps; the chain also equals the composition of
    its stages' closed forms on random input via explicit matrices."""
    rows = np.stack(_rows_for_pins()[:2])
    h = rng.standard_normal(23)
    N = 300
    hc = np.zeros(N)
    hc[0] = 1.0
    for r in rows:
        hc = np.convolve(hc, biquad_impulse_closed_form(r, N))[:N]
    want = np.convolve(hc, h)[:N]
    x = np.zeros(N)
    x[0] = 1.0
    got = lib.chain(x, [("sos", rows), ("fir", h)])
    assert _rel(got, want) < 1e-9
    # FIR first, then SOS: same impulse response (LTI), explicit check
    got2 = lib.chain(x, [("fir", h), ("sos", rows)])
    assert _rel(got2, want) < 1e-9
    # random input: y = T_chain x with T_chain the Toeplitz of the chain impulse response
    xs = rng.standard_normal(N)
    T = np.zeros((N, N))
    for i in range(N):
        T[i, : i + 1] = want[i::-1]
    got3 = lib.chain(xs, [("sos", rows), ("fir", h)])
    assert _rel(got3, T @ xs) < 1e-9


def pin_linearity_time_invariance(lib, rng):
    rows = np.stack(_rows_for_pins()[:3])
    h = rng.standard_normal(17)
    st = [("sos", rows), ("fir", h)]
    x1 = rng.standard_normal(400)
    x2 = rng.standard_normal(400)
    a, b = 0.7, -1.3
    lhs = lib.chain(a * x1 + b * x2, st)
    rhs = a * lib.chain(x1, st) + b * lib.chain(x2, st)
    assert _rel(lhs, rhs) < 1e-11
    k = 37
    xd = np.concatenate([np.zeros(k), x1[:-k]])
    yd = lib.chain(xd, st)
    y = lib.chain(x1, st)
    assert np.max(np.abs(yd[:k])) == 0.0
    assert _rel(yd[k:], y[:-k]) < 1e-12


def _vjp_case(rng):
    rows = np.stack(_rows_for_pins()[:2] + [_rows_for_pins()[6]])  # includes a0 != 1
    h = rng.standard_normal(7)
    stages = [("sos", rows[:2]), ("fir", h), ("sos", rows[2:])]
    x = rng.standard_normal((2, 60))
    g = rng.standard_normal((2, 60))
    return stages, x, g


def pin_vjp_finite_differences(lib, rng):
    """Coefficient gradients of L = sum(g * chain(x)) against central finite
    differences of the forward chain (step 1e-6, FP64)."""
    stages, x, g = _vjp_case(rng)
    _, grads = lib.chain_vjp(x, g, stages)
    eps = 1e-6
    for i, (kind, coef) in enumerate(stages):
        c = np.asarray(coef, dtype=np.float64)
        for idx in np.ndindex(c.shape):
            cp, cm = c.copy(), c.copy()
            cp[idx] += eps
            cm[idx] -= eps
            sp = list(stages)
            sp[i] = (kind, cp)
            sm = list(stages)
            sm[i] = (kind, cm)
            fd = (np.sum(g * lib.chain(x, sp)) - np.sum(g * lib.chain(x, sm))) / (2 * eps)
            got = grads[i][idx]
            assert abs(got - fd) <= 1e-6 * max(1.0, abs(fd)), f"stage {i} coef {idx}: {got} vs FD {fd}"


def pin_vjp_input_adjoint(lib, rng):
    """dL/dx is the adjoint of the chain: <g, chain(v)> = <dx(g), v> for any v,
    and matches central differences in x."""
    stages, x, g = _vjp_case(rng)
    dx, _ = lib.chain_vjp(x, g, stages)
    v = rng.standard_normal(x.shape)
    lhs = np.sum(g * lib.chain(v, stages))
    rhs = np.sum(dx * v)
    assert abs(lhs - rhs) <= 1e-10 * max(1.0, abs(lhs))
    eps = 1e-6
    for (c, m) in [(0, 0), (1, 17), (0, 59)]:
        xp, xm = x.copy(), x.copy()
        xp[c, m] += eps
        xm[c, m] -= eps
        fd = (np.sum(g * lib.chain(xp, stages)) - np.sum(g * lib.chain(xm, stages))) / (2 * eps)
        assert abs(dx[c, m] - fd) <= 1e-6 * max(1.0, abs(fd))


def pin_vjp_fir_definition(lib, rng):
    """Single FIR: dL/dh_k = sum_n g[n] x[n-k] (correlation, summed over channels)."""
    h = rng.standard_normal(9)
    x = rng.standard_normal((3, 40))
    g = rng.standard_normal((3, 40))
    _, (dh,) = lib.chain_vjp(x, g, [("fir", h)])
    want = np.array([sum(np.sum(g[c, k:] * x[c, :40 - k]) for c in range(3)) for k in range(9)])
    assert np.max(np.abs(dh - want)) <= 1e-12 * np.max(np.abs(want))


def pin_vjp_dx_sampled(lib, rng):
    """dL/dx at chosen samples (impulse-response route) against central
    differences of the forward chain in those samples."""
    stages, x, g = _vjp_case(rng)
    idx = [0, 5, 31, 59]
    got = lib.chain_vjp_dx_at(g[1], stages, idx)
    eps = 1e-6
    for m, v in zip(idx, got):
        xp, xm = x[1].copy(), x[1].copy()
        xp[m] += eps
        xm[m] -= eps
        fd = (np.sum(g[1] * lib.chain(xp, stages)) - np.sum(g[1] * lib.chain(xm, stages))) / (2 * eps)
        assert abs(v - fd) <= 1e-6 * max(1.0, abs(fd)), f"sample {m}: {v} vs FD {fd}"


ALL_PINS = [
    pin_fir_impulse,
    pin_fir_toeplitz,
    pin_fir_at_sampled,
    pin_fir_dc_nyquist,
    pin_sos_impulse_closed_form,
    pin_sos_steady_state,
    pin_sos_banded_solve,
    pin_sos_scale_invariance,
    pin_cascade_closed_form,
    pin_chain_closed_form,
    pin_linearity_time_invariance,
    pin_vjp_finite_differences,
    pin_vjp_input_adjoint,
    pin_vjp_fir_definition,
    pin_vjp_dx_sampled,
]
