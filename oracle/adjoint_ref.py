"""Exact transpose of the funnel transform (the map is linear in the image).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The forward operator A: img (H x W) -> P (H' x S) is the composition of the
four steps of Sec. 3.1 (see ``funnel_ref``), each linear over the reals.  For a
real loss and complex intermediates the gradient is carried as
dL/dRe + j dL/dIm; the transposes, taken in reverse order, are

* step 4: gG[l, m] = (c_l / H') sum_n g[n, m] exp(-j 2 pi l n / H')
* step 3: gV[l, x'] = sum_m gG[l, m] exp(-j 2 pi m x' / S)
* step 2: gF[l, x] = sum_{x'} w_l(x', x) gV[l, x']  (the interpolation weights
  scattered back to the columns they were gathered from; row 0 gets nothing)
* step 1: g_img[y, x] = sum_{l=0}^{H'/2} Re{gF[l, x] exp(+j 2 pi l y / H')},
  cropped to the rows of the original image (Sec. 4.2 padding).
"""
from __future__ import annotations

import numpy as np

from .transform import (centred, parity, nvmt_positions, interp_weights, dirichlet)


def adjoint_ref(g: np.ndarray, H: int, W: int, interp: str = "linear") -> np.ndarray:
    g = np.asarray(g, dtype=np.float64)
    Hp, S = g.shape
    L = Hp // 2 + 1
    l = np.arange(L)
    c = np.full(L, 2.0)
    c[0] = 1.0
    c[-1] = 1.0

    # step 4 transpose: numpy's FFT runs over t = n + H'/2, and
    # exp(-j 2 pi l n / H') = exp(-j 2 pi l t / H') (-1)^l
    gG = np.fft.rfft(g, axis=0) * (parity(l) * c / Hp)[:, None]

    # step 3 transpose: re-index m -> m mod S, then sum with exp(-j 2 pi m x'/S)
    m = centred(S)
    arr = np.zeros_like(gG)
    arr[:, m % S] = gG
    xp = centred(S)
    gV = np.fft.fft(arr, axis=1)[:, xp % S]

    # step 2 transpose: scatter the interpolation weights back
    gF = np.zeros((L, W), dtype=np.complex128)
    for li in range(1, L):
        i0, frac = nvmt_positions(li, S, Hp)
        if interp == "fourier":
            p = i0.astype(np.float64) + frac
            xs = centred(W).astype(np.float64)
            K = dirichlet(p[:, None] - xs[None, :], W)
            inside = (p >= -W // 2) & (p <= W // 2 - 1)
            gF[li] = (K * inside[:, None]).T @ gV[li]
            continue
        taps, w = interp_weights(i0, frac, interp)
        col = taps + W // 2
        ok = (col >= 0) & (col < W)
        np.add.at(gF[li], col[ok], (w * gV[li][:, None])[ok])

    # step 1 transpose over the expanded rows r = y + H'/2:
    # exp(+j 2 pi l y / H') = exp(+j 2 pi l r / H') (-1)^l; sum_l Re{X_l e^{..}}
    # equals H' * irfft(Y) with Y = X at l = 0, H'/2 and X/2 in between.
    X = gF * parity(l)[:, None]
    Y = X.copy()
    Y[1:-1] *= 0.5
    g_img_p = Hp * np.fft.irfft(Y, n=Hp, axis=0)
    top = (Hp - H) // 2
    return g_img_p[top:top + H]


def map_loss_grad_ref(P: np.ndarray, target: np.ndarray, W: int):
    """Loss of the gradient workload: mean((|P| / (W/2) - T)^2) and dL/dP.
    The derivative of |P| is taken as sign(P) (0 at P = 0)."""
    P = np.asarray(P, dtype=np.float64)
    scale = 2.0 / W
    r = np.abs(P) * scale - target
    loss = float(np.mean(r * r))
    dP = 2.0 * r * scale * np.sign(P) / P.size
    return loss, dP
