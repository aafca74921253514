"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of ``oracle/`` to something other than itself: an
explicit Fourier sum, a closed form derived by hand, a law the paper states
(line-to-point mapping eq. 19 with eqs. 22-23, point-to-line mapping eq. 13,
wrapping eqs. 20-21, the symmetry relation of Sec. 3.1), the worked example of
Fig. 9, or a brute-force enumeration on tiny inputs.  None of them runs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import transform as fr
from tests._lines import ridge_image, wrap_centred

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(20190419)


def explicit_dft(x, sign, coords_in, coords_out, n):
    """sum_u x[u] exp(sign j 2 pi k u / n) along axis 0, as a dense matrix."""
    Mx = np.exp(sign * 2j * np.pi * np.outer(coords_out, coords_in) / n)
    return Mx @ x


# ---------------------------------------------------------------- FFT stages
def test_step1_matches_explicit_sum_32x32():
    img = RNG.standard_normal((32, 32))
    Hp = 32
    F = fr.fourier_y(img)
    y = np.arange(Hp) - Hp // 2
    ref = explicit_dft(img, -1, y, np.arange(Hp // 2 + 1), Hp)
    np.testing.assert_allclose(F, ref, rtol=0, atol=1e-11)


def test_step3_matches_explicit_sum():
    S = 32
    V = RNG.standard_normal((5, S)) + 1j * RNG.standard_normal((5, S))
    G = fr.fourier_xprime(V)
    c = np.arange(S) - S // 2
    ref = explicit_dft(V.T, +1, c, c, S).T
    np.testing.assert_allclose(G, ref, rtol=0, atol=1e-11)


def test_step4_matches_explicit_real_sum():
    Hp, S = 24, 6
    L = Hp // 2 + 1
    G = RNG.standard_normal((L, S)) + 1j * RNG.standard_normal((L, S))
    P = fr.inverse_fourier_omega2(G, Hp)
    n = np.arange(Hp) - Hp // 2
    ref = np.zeros((Hp, S))
    for l in range(L):
        c = 1.0 if l in (0, Hp // 2) else 2.0
        ref += c * np.real(G[l][None, :] * np.exp(2j * np.pi * l * n / Hp)[:, None])
    np.testing.assert_allclose(P, ref / Hp, rtol=0, atol=1e-12)


def test_parseval_each_stage():
    H, W, S, Hp = 20, 16, 24, 28
    img = RNG.standard_normal((H, W))
    P, F, V, G = fr.funnel_ref(img, S, Hp, return_stages=True)
    # step 1: real input, half spectrum
    e_img = Hp * np.sum(img ** 2)
    e_F = np.sum(np.abs(F[0]) ** 2) + np.sum(np.abs(F[-1]) ** 2) + 2 * np.sum(np.abs(F[1:-1]) ** 2)
    assert abs(e_img - e_F) <= 1e-11 * e_img
    # step 3: full complex DFT of each row
    assert abs(np.sum(np.abs(G) ** 2) - S * np.sum(np.abs(V) ** 2)) <= 1e-11 * np.sum(np.abs(G) ** 2)
    # step 4: real output whose half spectrum is G with real end bins
    e_P = Hp * np.sum(P ** 2)
    e_G = np.sum(G[0].real ** 2) + np.sum(G[-1].real ** 2) + 2 * np.sum(np.abs(G[1:-1]) ** 2)
    assert abs(e_P - e_G) <= 1e-11 * e_G


# ----------------------------------------------------- whole map vs brute force
@pytest.mark.parametrize("interp", ["linear", "cubic", "fourier"])
@pytest.mark.parametrize("H,W,S,Hp", [(8, 8, 8, 8), (6, 8, 10, 12), (8, 6, 8, 10), (12, 10, 16, 14),
                                      (4, 2, 2, 6)])
def test_map_matches_direct_definition(H, W, S, Hp, interp):
    img = RNG.standard_normal((H, W))
    P = fr.funnel_ref(img, S, Hp, interp)
    D = oracle.funnel_direct(img, S, Hp, interp)
    scale = np.abs(P).max()
    assert np.abs(D.imag).max() <= 1e-12 * scale
    np.testing.assert_allclose(P, D.real, rtol=0, atol=1e-12 * scale)


def test_reversal_relation_negative_frequencies():
    """Sec. 3.1: for w2 < 0 the NVMT also reverses x', so that
    V(x', w2) = conj V(-x', -w2); computed here from the explicit negative-
    frequency spectrum and the NVMT position x' H' / (2 l) with l < 0."""
    H, W, S, Hp = 10, 12, 16, 14
    img = RNG.standard_normal((H, W))
    F = fr.fourier_y(fr.pad_rows(img, Hp))
    y = np.arange(Hp) - Hp // 2
    xs = np.arange(W) - W // 2
    xps = np.arange(S) - S // 2
    for l in range(1, Hp // 2 + 1):
        Fneg = np.exp(+2j * np.pi * l * y / Hp) @ fr.pad_rows(img, Hp)     # row -l
        p = xps * Hp / (2.0 * -l)
        hat = np.maximum(0.0, 1.0 - np.abs(p[:, None] - xs[None, :]))
        Vneg = hat @ Fneg
        Vpos = fr.nvmt_row(F[l], l, S, Hp, "linear")
        for i, xp in enumerate(xps):
            if xp == -S // 2:
                continue                         # -x' = S/2 is outside the stored range
            j = int(np.where(xps == -xp)[0][0])
            assert abs(Vneg[i] - np.conj(Vpos[j])) <= 1e-10 * (1 + abs(Vpos[j]))


def test_nyquist_row_is_identity_resampling():
    """At l = H'/2 the NVMT samples x = x' exactly, for every interpolator."""
    H, W, S, Hp = 12, 10, 14, 12
    img = RNG.standard_normal((H, W))
    F = fr.fourier_y(fr.pad_rows(img, Hp))
    for interp in ("linear", "cubic", "fourier"):
        V = fr.nvmt(F, S, Hp, interp)
        ref = np.zeros(S, dtype=complex)
        ref[S // 2 - W // 2:S // 2 + W // 2] = F[-1]
        np.testing.assert_allclose(V[-1], ref, atol=1e-10)
        assert np.all(V[0] == 0)


@pytest.mark.parametrize("which", ["transform.keys_cubic", "funnel_direct._keys"])
def test_keys_kernel_properties(which):
    """Keys' kernel with a = -1/2 (the cubic interpolator of step 2), in both
    oracle forms: interpolating, even, support |s| < 2, partition of unity,
    exact on linear and quadratic sequences, C1 at |s| = 0, 1, 2, and equal
    to the Catmull-Rom spline (midpoint weights -1/16, 9/16, 9/16, -1/16)."""
    import importlib
    from tests._keys import keys_failures
    fd = importlib.import_module("oracle.funnel_direct")
    k = fr.keys_cubic if which.startswith("transform") else np.vectorize(fd._keys)
    assert keys_failures(k) == []


def test_cubic_nvmt_row_is_catmull_rom_and_exact_on_quadratics():
    """Step 2 with the cubic interpolator: wherever the four taps lie inside the
    row, the sample at p = x' H' / (2 l) is the Catmull-Rom spline through the
    row at p, and a quadratic row a + b x + c x^2 comes out as a + b p + c p^2."""
    from tests._keys import catmull_rom
    W, S, Hp = 24, 40, 36
    xs = np.arange(W) - W // 2
    row = RNG.standard_normal(W) + 1j * RNG.standard_normal(W)
    quad = 0.3 - 1.7 * xs + 0.25 * xs ** 2 + 0j
    checked = 0
    for l in (5, 9, 13, 18):
        i0, frac = fr.nvmt_positions(l, S, Hp)
        V = fr.nvmt_row(row, l, S, Hp, "cubic")
        Q = fr.nvmt_row(quad, l, S, Hp, "cubic")
        inside = (i0 - 1 >= -W // 2) & (i0 + 2 <= W // 2 - 1)
        checked += int(inside.sum())
        c = i0 + W // 2
        for j in np.flatnonzero(inside):
            cr = catmull_rom(row[c[j] - 1], row[c[j]], row[c[j] + 1], row[c[j] + 2], frac[j])
            assert abs(V[j] - cr) <= 1e-12
            p = (j - S // 2) * Hp / (2.0 * l)
            assert abs(Q[j] - (0.3 - 1.7 * p + 0.25 * p * p)) <= 1e-9
    assert checked >= 40


def test_linearity():
    H, W, S, Hp = 16, 16, 20, 24
    a, b = RNG.standard_normal((2, H, W))
    lhs = fr.funnel_ref(2.5 * a - 0.75 * b, S, Hp)
    rhs = 2.5 * fr.funnel_ref(a, S, Hp) - 0.75 * fr.funnel_ref(b, S, Hp)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12 * np.abs(lhs).max())


def test_nvmt_positions_exact():
    """x' H' / (2 l) split into floor and fraction exactly (checked with Fraction)."""
    from fractions import Fraction
    for (S, Hp, l) in [(16, 24, 5), (30, 18, 7), (12, 12, 6), (64, 96, 1)]:
        i0, f = fr.nvmt_positions(l, S, Hp)
        for xp, a, b in zip(np.arange(S) - S // 2, i0, f):
            p = Fraction(int(xp) * Hp, 2 * l)
            assert int(a) == math.floor(p)
            assert b == float(p - math.floor(p))


# --------------------------------------------------------------- closed forms
@pytest.mark.parametrize("S,Hp,y0", [(16, 16, 3), (20, 24, -5), (16, 32, 0)])
def test_horizontal_line_closed_form(S, Hp, y0):
    """img = 1 on the row y = y0.  Then F[l, x] = exp(-j 2 pi l y0 / H') on every
    column, V[l, x'] = exp(-j 2 pi l y0 / H') sigma_l(x') with sigma_l the hat-
    interpolated column indicator, and the m = 0 column of the map is
    (1/H') sum_l c_l |supp_l| cos(2 pi l (n - y0) / H'), |supp_l| = sum sigma_l."""
    H, W = Hp // 2, 16 if S >= 16 else S
    top = (Hp - H) // 2
    img = np.zeros((H, W))
    img[y0 + Hp // 2 - top, :] = 1.0
    P = fr.funnel_ref(img, S, Hp)
    xs = np.arange(W) - W // 2
    n = np.arange(Hp) - Hp // 2
    col = np.zeros(Hp)
    for l in range(1, Hp // 2 + 1):
        supp = 0.0
        for xp in range(-S // 2, S // 2):
            p = xp * Hp / (2.0 * l)
            supp += sum(max(0.0, 1.0 - abs(p - x)) for x in xs)
        c = 1.0 if l == Hp // 2 else 2.0
        col += c * supp * np.cos(2 * np.pi * l * (n - y0) / Hp)
    col /= Hp
    np.testing.assert_allclose(P[:, S // 2], col, atol=1e-12 * np.abs(col).max())
    t, s = np.unravel_index(np.argmax(np.abs(P)), P.shape)
    assert (s, t) == (S // 2, y0 + Hp // 2)


@pytest.mark.parametrize("Hp", [64, 128])
def test_line_to_point_mapping(Hp):
    """Eq. (19) with eqs. (22)-(23): a line y = k x + b becomes one peak at
    m = k S / 2, n = b."""
    H = W = S = 64
    for k in np.linspace(-0.9, 0.9, 7):
        for b in (-20.0, -5.0, 0.0, 7.0, 19.0):
            P = fr.funnel_ref(ridge_image(H, W, Hp, [(k, b)]), S, Hp)
            t, s = np.unravel_index(np.argmax(np.abs(P)), P.shape)
            m, n = s - S // 2, t - Hp // 2
            assert abs(m - k * S / 2) <= 0.5 + 1e-9, (k, b, m, n)
            assert abs(n - b) <= 1, (k, b, m, n)


def test_line_to_point_with_zero_insertion():
    """n_slope > W refines the slope grid (Sec. 4.3): k = 2 m / S still holds."""
    H = W = 48
    S, Hp = 96, 96
    for k, b in [(0.5, 3.0), (-0.75, -10.0), (0.25, 12.0)]:
        P = fr.funnel_ref(ridge_image(H, W, Hp, [(k, b)]), S, Hp)
        t, s = np.unravel_index(np.argmax(np.abs(P)), P.shape)
        assert abs((s - S // 2) - k * S / 2) <= 1.0
        assert abs((t - Hp // 2) - b) <= 1


def test_point_to_line_mapping():
    """Eq. (13): a point (u, v) becomes the line y = v + (u / w_max) w1 in the
    map; with w1 = -2 pi m / S (the exp(+j) kernel of step 3) and w_max = pi this
    is n = v - 2 u m / S.  The NVMT samples that line only at integer x', so the
    column-wise maximum sits within half a cell of it on most columns and within
    1.5 cells where the line crosses a half-integer n (two cells then share the
    response).  The column m = -S/2 is skipped: slopes +-1 alias there."""
    H = W = S = 64
    Hp = 128
    for (u, v) in [(6, -9), (3, 5), (-10, 20), (12, 0)]:
        top = (Hp - H) // 2
        img = np.zeros((H, W))
        img[v + Hp // 2 - top, u + W // 2] = 1.0
        A = np.abs(fr.funnel_ref(img, S, Hp))
        errs = []
        for m in range(-S // 2 + 1, S // 2):
            t = int(np.argmax(A[:, m + S // 2]))
            n_expect = wrap_centred(v - 2.0 * u * m / S, Hp)
            errs.append(abs(wrap_centred((t - Hp // 2) - n_expect, Hp)))
        errs = np.array(errs)
        assert errs.max() <= 1.5 + 1e-9, (u, v, errs.max())
        assert np.mean(errs <= 0.5 + 1e-9) >= 0.85, (u, v)


def test_intercept_wrap_eq20():
    """Eq. (20): without expansion (H' = H) an intercept outside (-H/2, H/2]
    appears at b - H p."""
    H = W = S = Hp = 64
    for k, b in [(0.75, 38.0), (-0.75, -38.0), (0.5, 36.0), (1.0, 34.0)]:
        # |b| > H/2: the line crosses the image only where |k x + b| < H/2
        # (24-30 of the 64 columns for these cases)
        P = fr.funnel_ref(ridge_image(H, W, Hp, [(k, b)]), S, Hp)
        t, s = np.unravel_index(np.argmax(np.abs(P)), P.shape)
        assert abs(wrap_centred((t - Hp // 2) - b, Hp)) <= 1
        # only part of the line is inside; k = 1 sits on m = -S/2 = +S/2 (eq. 21)
        assert abs(wrap_centred((s - S // 2) - k * S / 2, S)) <= 1.0


def test_slope_wrap_eq21():
    """Eq. (21) / Fig. 7: a line of slope k = 2 q + k~ peaks at the slope k~ in (-1, 1]."""
    H, W = 96, 64
    Hp, S = 160, 64
    for k in (math.sqrt(3.0), 1.5, -1.4):
        kt = k - 2.0 * round(k / 2.0)
        P = fr.funnel_ref(ridge_image(H, W, Hp, [(k, 0.0)]), S, Hp)
        t, s = np.unravel_index(np.argmax(np.abs(P)), P.shape)
        assert abs((s - S // 2) - kt * S / 2) <= 1.0, (k, kt, s - S // 2)
        assert abs(t - Hp // 2) <= 1


def test_fig9_worked_example():
    with open(os.path.join(GOLDEN, "fig9_wrapped_peak.json")) as f:
        g = json.load(f)
    W, H, k = g["width_M"], g["height_N"], g["slope_k"]
    Hp = g["expanded_length"]
    tol = g["tolerance_cells"]
    m_r, n_r = g["regular_peak_mn"]
    img = ridge_image(H, W, Hp, [(k, float(n_r))])
    A = np.abs(fr.funnel_ref(img, W, Hp))
    t, s = np.unravel_index(np.argmax(A), A.shape)
    assert abs((s - W // 2) - m_r) <= tol and abs((t - Hp // 2) - n_r) <= tol
    # the unwrapped peak in the inverse (dual) space, eqs. (24)-(25)
    m_i, n_i = g["inverse_peak_mn"]
    Q = np.abs(oracle.inverse_funnel_ref(img, H, W + H))
    t, s = np.unravel_index(np.argmax(Q), Q.shape)
    assert abs((t - (W + H) // 2) - m_i) <= tol and abs((s - H // 2) - n_i) <= tol
    inv_k, b_x = oracle.inverse_peak_to_line(t, s, H, W + H)
    assert abs(1.0 / inv_k - k) < 0.1


# ------------------------------------------------------------------- peaks
def brute_local_max_topk(A, K, T=-np.inf):
    """Strict local maxima of the wrap-around 3x3 neighbourhood under the total
    order (value desc, linear index asc), sorted by that order, value >= T."""
    Hp, S = A.shape
    key = lambda t, s: (-A[t, s], t * S + s)
    cands = []
    for t in range(Hp):
        for s in range(S):
            if A[t, s] < T:
                continue
            ok = True
            for dt in (-1, 0, 1):
                for ds in (-1, 0, 1):
                    tt, ss = (t + dt) % Hp, (s + ds) % S
                    if (tt, ss) != (t, s) and key(tt, ss) < key(t, s):
                        ok = False
            if ok:
                cands.append(key(t, s))
    cands.sort()
    return [(lin // S, lin % S) for _, lin in cands[:K]]


@pytest.mark.parametrize("shape", [(2, 2), (4, 6), (8, 8), (6, 10), (16, 12)])
def test_peak_list_equals_local_max_form(shape):
    for trial in range(20):
        A = RNG.integers(0, 4, size=shape).astype(float)     # many ties on purpose
        for K in (1, 3, 50):
            for T in (-np.inf, 1.0, 2.0):
                got = [(t, s) for t, s, _ in oracle.peaks_ref(A, K, T)]
                assert got == brute_local_max_topk(A, K, T)


def test_peak_list_continuous_values():
    A = RNG.random((32, 32))
    got = [(t, s) for t, s, _ in oracle.peaks_ref(A, 40)]
    assert got == brute_local_max_topk(A, 40)


def test_peak_to_line_eq22_23():
    assert oracle.peak_to_line(0, 0, 256, 512) == (-1.0, -256.0)
    assert oracle.peak_to_line(256, 128, 256, 512) == (0.0, 0.0)
    assert oracle.peak_to_line(300, 192, 256, 512) == (0.5, 44.0)


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("interp", ["linear", "cubic", "fourier"])
@pytest.mark.parametrize("H,W,S,Hp", [(10, 12, 16, 18), (16, 16, 16, 16), (8, 6, 12, 20)])
def test_adjoint_dot_product(H, W, S, Hp, interp):
    x = RNG.standard_normal((H, W))
    y = RNG.standard_normal((Hp, S))
    a = np.sum(fr.funnel_ref(x, S, Hp, interp) * y)
    b = np.sum(x * oracle.adjoint_ref(y, H, W, interp))
    assert abs(a - b) <= 1e-12 * max(abs(a), 1.0)


def test_adjoint_equals_explicit_transpose():
    H, W, S, Hp = 6, 4, 6, 8
    A = np.zeros((Hp * S, H * W))
    for j in range(H * W):
        e = np.zeros(H * W)
        e[j] = 1.0
        A[:, j] = fr.funnel_ref(e.reshape(H, W), S, Hp).ravel()
    y = RNG.standard_normal((Hp, S))
    np.testing.assert_allclose(oracle.adjoint_ref(y, H, W).ravel(), A.T @ y.ravel(), atol=1e-12)


def test_loss_gradient_central_differences_64():
    """Gradient of mean((|P|/(W/2) - T)^2) through the adjoint vs FP64 central
    differences (step 1e-6) on a 64 x 64 image."""
    H = W = S = Hp = 64
    img = ridge_image(H, W, Hp, [(0.3, 5.0), (-0.6, -12.0)]) + 0.05 * RNG.standard_normal((H, W))
    target = np.zeros((Hp, S))
    target[5 + Hp // 2, int(round(0.3 * S / 2)) + S // 2] = 1.0
    P = fr.funnel_ref(img, S, Hp)
    _, dP = oracle.map_loss_grad_ref(P, target, W)
    grad = oracle.adjoint_ref(dP, H, W)
    idx = [(3, 4), (32, 32), (40, 10), (63, 63), (0, 17), (20, 50), (31, 2), (50, 45)]
    h = 1e-6
    fd = []
    for (r, c) in idx:
        e = np.zeros_like(img)
        e[r, c] = h
        lp, _ = oracle.map_loss_grad_ref(fr.funnel_ref(img + e, S, Hp), target, W)
        lm, _ = oracle.map_loss_grad_ref(fr.funnel_ref(img - e, S, Hp), target, W)
        fd.append((lp - lm) / (2 * h))
    fd = np.array(fd)
    an = np.array([grad[r, c] for r, c in idx])
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an)
