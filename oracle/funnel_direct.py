"""Brute-force evaluation of the funnel-transform definition (tiny sizes only).

TEST INFRASTRUCTURE ONLY.  This is a second, independent evaluation of the
definition written out in the docstring of ``oracle.transform`` (Sec. 3.1 steps 1-4,
eqs. 16-19, Sec. 4.2): every Fourier sum is an explicit loop over exponentials
(no FFT), every NVMT sample position x' H' / (2 l) is an exact fraction, the
interpolators are written as kernels of the distance p - x (hat function,
Keys cubic, trigonometric sum), and the inverse along w2 is the two-sided sum
over l = -H'/2 .. H'/2 with the end points weighted 1/2 and the negative half
taken as the complex conjugate of the positive half (the symmetry relation of
Sec. 3.1).  The result is returned complex so that tests can check it is real.
"""
from __future__ import annotations

import cmath
import math
from fractions import Fraction

import numpy as np

KEYS_A = -0.5


def _hat(d: float) -> float:
    return max(0.0, 1.0 - abs(d))


def _keys(d: float) -> float:
    a, s = KEYS_A, abs(d)
    if s <= 1.0:
        return (a + 2.0) * s ** 3 - (a + 3.0) * s ** 2 + 1.0
    if s < 2.0:
        return a * s ** 3 - 5.0 * a * s ** 2 + 8.0 * a * s - 4.0 * a
    return 0.0


def _trig_interp(row: list, p: float) -> complex:
    """Trigonometric interpolant of the periodic length-W sequence ``row`` (index
    c = x + W/2) at real position p (centred), Nyquist term as a cosine."""
    W = len(row)
    xs = [c - W // 2 for c in range(W)]
    total = 0j
    for u in range(-W // 2 + 1, W // 2):
        coef = sum(row[c] * cmath.exp(-2j * math.pi * u * xs[c] / W) for c in range(W))
        total += coef * cmath.exp(2j * math.pi * u * p / W)
    nyq = sum(row[c] * cmath.exp(-1j * math.pi * xs[c]) for c in range(W))
    total += nyq * math.cos(math.pi * p)
    return total / W


def funnel_direct(img, n_slope: int | None = None, n_intercept: int | None = None,
                  interp: str = "linear") -> np.ndarray:
    img = np.asarray(img, dtype=np.float64)
    H, W = img.shape
    S = W if n_slope is None else int(n_slope)
    Hp = H if n_intercept is None else int(n_intercept)
    top = (Hp - H) // 2
    ys = [r + top - Hp // 2 for r in range(H)]          # centred y of each image row
    xs = [c - W // 2 for c in range(W)]                 # centred x of each column
    xps = [i - S // 2 for i in range(S)]                # centred x'
    ms = [i - S // 2 for i in range(S)]                 # centred slope index m
    ns = [i - Hp // 2 for i in range(Hp)]               # centred intercept index n

    G = {}
    for l in range(1, Hp // 2 + 1):
        # step 1: explicit Fourier sum along y at w2 = 2 pi l / H'
        F = [sum(img[r, c] * cmath.exp(-2j * math.pi * l * ys[r] / Hp) for r in range(H))
             for c in range(W)]
        # step 2: NVMT, sample x = x' H' / (2 l) exactly
        V = []
        for xp in xps:
            p = Fraction(xp * Hp, 2 * l)
            pf = float(p)
            if interp == "linear":
                V.append(sum(_hat(pf - xs[c]) * F[c] for c in range(W)))
            elif interp == "cubic":
                V.append(sum(_keys(pf - xs[c]) * F[c] for c in range(W)))
            elif interp == "fourier":
                inside = Fraction(-W, 2) <= p <= Fraction(W, 2) - 1
                V.append(_trig_interp(F, pf) if inside else 0j)
            else:
                raise ValueError(interp)
        # step 3: explicit Fourier sum along x' with the exp(+j) kernel
        G[l] = [sum(V[i] * cmath.exp(2j * math.pi * m * xps[i] / S) for i in range(S))
                for m in ms]

    P = np.zeros((Hp, S), dtype=np.complex128)
    for ti, n in enumerate(ns):
        for si in range(S):
            acc = 0j
            for l in range(1, Hp // 2 + 1):
                w = 0.5 if l == Hp // 2 else 1.0
                g = G[l][si]
                acc += w * g * cmath.exp(2j * math.pi * l * n / Hp)
                acc += w * g.conjugate() * cmath.exp(-2j * math.pi * l * n / Hp)
            P[ti, si] = acc / Hp
    return P
