"""FP64 reference of the regular funnel transform, step by step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the CUDA library never
imports this module and this module imports nothing from the library.

Definition followed (Wei, Feng & Zheng, "Funnel Transform for Straight Line
Detection"):

* Sec. 4.2 (Fig. 6): the M x N image (width M, height N) is expanded with zero
  rows above and below.  For a general intercept length H' >= H the oracle puts
  (H'-H)//2 zero rows above and the rest below.  The coordinate origin is the
  centre of the expanded image: x = col - W/2, y = row_p - H'/2.
* Sec. 3.1, step 1, eq. (16): F(x, w2) = sum_y I(x, y) exp(-j w2 y), sampled at
  w2 = 2 pi l / H'.  Because I is real, F(x, -w2) = conj F(x, w2), so only
  l = 0 .. H'/2 is kept.
* Sec. 3.1, step 2, eqs. (17)-(18): the nonlinear variable-metric transform
  (NVMT) x' = (w2 / w_max) x, i.e. the output sample x' reads row l at
  x = x' w_max / w2 = x' H' / (2 l) with w_max = pi.  Rows are interpolated in
  1D (linear, Keys cubic, or band-limited / chirp-z style), zero outside the
  image columns.  Row l = 0 is set to zero.
* Sec. 3.1, step 3: G(w1, w2) = sum_x' V(x', w2) exp(+j 2 pi m x' / S) over the
  centred x' in [-S/2, S/2), output m in [-S/2, S/2).
* Sec. 3.1, step 4, eq. (19): inverse transform along w2.  The negative half is
  the conjugate of the positive half with x' reversed (the relation
  V(x', w2) = conj V(-x', -w2) of Sec. 3.1), which makes the map real:
  P[n, m] = (1/H') sum_{l=0}^{H'/2} c_l Re{G[l, m] exp(+j 2 pi l n / H')},
  c_0 = c_{H'/2} = 1, c_l = 2 otherwise, n in [-H'/2, H'/2).
* Sec. 4.3, eqs. (22)-(23): peak (m, n) <-> line y = k x + b with k = 2 m / S,
  b = n.

Readings where the paper is silent or garbled: w_max = pi (the only value for
which eq. (22) holds with w2 = 2 pi l / H'); the exp(+j) kernel along x' (so
that the peak of y = kx + b sits at m = +kS/2 as eq. (22) states, where
eq. (19) would give the opposite sign); the centre origin with even sizes as
above; the DC row set to zero (the NVMT Jacobian |w2|/w_max vanishes there);
the Nyquist row enters through its real part; forward transforms are
unnormalised and the last inverse carries 1/H'.

The map is stored as ``P[t, s]`` with ``t = n + H'/2`` and ``s = m + S/2``.
"""
from __future__ import annotations

import numpy as np

INTERPS = ("linear", "cubic", "fourier")
KEYS_A = -0.5


def centred(n: int) -> np.ndarray:
    """Centred integer coordinates -n/2 .. n/2-1 of an even-length axis."""
    return np.arange(n, dtype=np.int64) - n // 2


def parity(idx: np.ndarray) -> np.ndarray:
    """(-1)^idx as float64 for integer arrays (negative entries allowed)."""
    return np.where(np.asarray(idx) % 2 == 0, 1.0, -1.0)


def pad_rows(img: np.ndarray, n_intercept: int) -> np.ndarray:
    """Sec. 4.2: expand an H x W image to n_intercept rows with zero rows,
    (n_intercept - H)//2 above and the rest below."""
    H, W = img.shape
    if n_intercept < H:
        raise ValueError("n_intercept must be >= image height")
    out = np.zeros((n_intercept, W), dtype=np.float64)
    top = (n_intercept - H) // 2
    out[top:top + H] = img
    return out


def fourier_y(img_p: np.ndarray) -> np.ndarray:
    """Step 1 (Sec. 3.1, eq. 16): F[l, x] = sum_y img_p[y, x] exp(-j 2 pi l y / H'),
    y = row - H'/2 centred, for l = 0 .. H'/2.  Returns (H'/2+1, W) complex128.

    numpy's FFT sums over the row index r = y + H'/2; since
    exp(-j 2 pi l y / H') = exp(-j 2 pi l r / H') * exp(+j pi l), the centred
    spectrum is numpy's spectrum times (-1)^l.
    """
    Hp = img_p.shape[0]
    L = Hp // 2 + 1
    l = np.arange(L)
    spec = np.fft.fft(np.asarray(img_p, dtype=np.float64), axis=0)[:L]
    return spec * parity(l)[:, None]


def nvmt_positions(l: int, n_slope: int, n_intercept: int):
    """Sampling positions of row l under the NVMT x = x' H' / (2 l) (eq. 17 with
    w_max = pi), as an exact integer floor i0 and a float64 fraction f in [0, 1).
    x' runs over the centred range [-S/2, S/2)."""
    if l <= 0:
        raise ValueError("the NVMT is defined for l >= 1")
    xp = centred(n_slope)
    num = xp * np.int64(n_intercept)
    den = np.int64(2 * l)
    i0 = np.floor_divide(num, den)
    frac = (num - i0 * den).astype(np.float64) / float(den)
    return i0, frac


def keys_cubic(s: np.ndarray, a: float = KEYS_A) -> np.ndarray:
    """Keys' cubic convolution kernel with parameter a."""
    s = np.abs(s)
    out = np.zeros_like(s)
    m1 = s <= 1.0
    m2 = (s > 1.0) & (s < 2.0)
    out[m1] = (a + 2.0) * s[m1] ** 3 - (a + 3.0) * s[m1] ** 2 + 1.0
    out[m2] = a * s[m2] ** 3 - 5.0 * a * s[m2] ** 2 + 8.0 * a * s[m2] - 4.0 * a
    return out


def interp_weights(i0: np.ndarray, frac: np.ndarray, interp: str):
    """Taps (centred x, shape (S, T)) and weights (S, T) of a local interpolator."""
    if interp == "linear":
        taps = np.stack([i0, i0 + 1], axis=1)
        w = np.stack([1.0 - frac, frac], axis=1)
    elif interp == "cubic":
        taps = np.stack([i0 - 1, i0, i0 + 1, i0 + 2], axis=1)
        w = np.stack([keys_cubic(frac + 1.0), keys_cubic(frac),
                      keys_cubic(1.0 - frac), keys_cubic(2.0 - frac)], axis=1)
    else:
        raise ValueError(f"no local taps for interp={interp!r}")
    return taps, w


def dirichlet(d: np.ndarray, W: int) -> np.ndarray:
    """Band-limited interpolation kernel of a length-W periodic sequence (even W),
    the Nyquist term taken as a cosine: (1/W)[1 + 2 sum_{u=1}^{W/2-1} cos(2 pi u d / W)
    + cos(pi d)].  At integer d it is 1 for d = 0 (mod W) and 0 otherwise."""
    d = np.asarray(d, dtype=np.float64)
    acc = np.ones_like(d) + np.cos(np.pi * d)
    for u in range(1, W // 2):
        acc += 2.0 * np.cos(2.0 * np.pi * u * d / W)
    return acc / W


def nvmt_row(F_row: np.ndarray, l: int, n_slope: int, n_intercept: int,
             interp: str) -> np.ndarray:
    """Step 2 for one row l >= 1: V[x'] = interpolated F_row at x = x' H' / (2 l).
    F_row is indexed by column c = x + W/2; outside x in [-W/2, W/2-1] it is zero."""
    W = F_row.shape[0]
    i0, frac = nvmt_positions(l, n_slope, n_intercept)
    if interp == "fourier":
        p = i0.astype(np.float64) + frac
        xs = centred(W).astype(np.float64)
        K = dirichlet(p[:, None] - xs[None, :], W)
        inside = (p >= -W // 2) & (p <= W // 2 - 1)
        return np.where(inside, K @ F_row, 0.0)
    taps, w = interp_weights(i0, frac, interp)
    col = taps + W // 2
    ok = (col >= 0) & (col < W)
    vals = F_row[np.clip(col, 0, W - 1)]
    return np.sum(np.where(ok, w * vals, 0.0), axis=1)


def nvmt(F: np.ndarray, n_slope: int, n_intercept: int, interp: str = "linear") -> np.ndarray:
    """Step 2 (Sec. 3.1, eqs. 17-18) on every kept row: V[l, x'] for
    l = 0 .. H'/2, x' = -S/2 .. S/2-1 (stored at x' + S/2).  V[0, :] = 0."""
    if interp not in INTERPS:
        raise ValueError(f"interp must be one of {INTERPS}")
    L = F.shape[0]
    V = np.zeros((L, n_slope), dtype=np.complex128)
    for l in range(1, L):
        V[l] = nvmt_row(F[l], l, n_slope, n_intercept, interp)
    return V


def fourier_xprime(V: np.ndarray) -> np.ndarray:
    """Step 3 (Sec. 3.1): G[l, m] = sum_{x'} V[l, x'] exp(+j 2 pi m x' / S),
    x' and m centred.  numpy's inverse FFT sums over i = x' + S/2 with
    exp(+j 2 pi q i / S); exp(+j 2 pi m x'/S) = exp(+j 2 pi m i / S) (-1)^m."""
    S = V.shape[1]
    m = centred(S)
    Y = S * np.fft.ifft(V, axis=1)
    return Y[:, m % S] * parity(m)[None, :]


def inverse_fourier_omega2(G: np.ndarray, n_intercept: int) -> np.ndarray:
    """Step 4 (Sec. 3.1, eq. 19): P[n, m] = (1/H') sum_{l=0}^{H'/2} c_l
    Re{G[l, m] exp(+j 2 pi l n / H')} with n centred.  numpy's irfft evaluates
    exactly this sum over the output index r = n + H'/2 (it keeps only the real
    parts of the DC and Nyquist bins), and exp(+j 2 pi l n / H') =
    exp(+j 2 pi l r / H') (-1)^l."""
    L = G.shape[0]
    l = np.arange(L)
    return np.fft.irfft(G * parity(l)[:, None], n=n_intercept, axis=0)


def funnel_ref(img: np.ndarray, n_slope: int | None = None, n_intercept: int | None = None,
               interp: str = "linear", return_stages: bool = False):
    """The regular funnel transform of one H x W image: returns the real map
    P[t, s] (n_intercept x n_slope, float64).  With ``return_stages`` also the
    intermediate F (step 1), V (step 2) and G (step 3)."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    S = W if n_slope is None else int(n_slope)
    Hp = H if n_intercept is None else int(n_intercept)
    if S % 2 or Hp % 2 or W % 2 or S < W or Hp < H:
        raise ValueError("need even W, n_slope >= W and even n_intercept >= H")
    img_p = pad_rows(img, Hp)
    F = fourier_y(img_p)
    V = nvmt(F, S, Hp, interp)
    G = fourier_xprime(V)
    P = inverse_fourier_omega2(G, Hp)
    if return_stages:
        return P, F, V, G
    return P


def inverse_funnel_ref(img: np.ndarray, n_inv_slope: int | None = None,
                       n_x_intercept: int | None = None, interp: str = "linear"):
    """The dual (inverse) funnel transform of Sec. 3.1: Fourier transform along x,
    NVMT y' = (w1 / w_max) y, Fourier transform along y', inverse along w1.
    With x and y exchanged this is the regular transform of the transposed image;
    the returned map Q[t, s] has t = b_x + W'/2 (x-intercept, eq. 25) and
    s = n + S'/2 with 1/k = 2 n / S' (eq. 24)."""
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    return funnel_ref(img.T, H if n_inv_slope is None else n_inv_slope,
                      W if n_x_intercept is None else n_x_intercept, interp)
