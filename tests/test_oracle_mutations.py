"""Planted mistakes in the oracle must be caught by its pins.

Each case swaps one step of ``oracle.transform`` for a plausible wrong version
(a flipped sign, a dropped term, a transposed index, an inverted scale) on the
CPU and checks that the brute-force comparison or the line-to-point law no
longer holds.  This shows that the pins in ``test_oracle_pins`` can fail.
"""
import numpy as np
import pytest

import oracle
from oracle import transform as fr
from tests._lines import ridge_image


def _wrong_sign_step3(V):
    S = V.shape[1]
    m = fr.centred(S)
    Y = np.fft.fft(V, axis=1)                  # exp(-j) instead of exp(+j)
    return Y[:, m % S] * fr.parity(m)[None, :]


def _no_centring_step1(img_p):
    Hp = img_p.shape[0]
    return np.fft.fft(img_p, axis=0)[: Hp // 2 + 1]


def _inverted_nvmt_positions(l, n_slope, n_intercept):
    xp = fr.centred(n_slope)
    num = xp * np.int64(2 * l)                  # x' 2l / H' instead of x' H' / (2l)
    den = np.int64(n_intercept)
    i0 = np.floor_divide(num, den)
    return i0, (num - i0 * den).astype(np.float64) / float(den)


def _pad_all_above(img, n_intercept):
    H, W = img.shape
    out = np.zeros((n_intercept, W))
    out[n_intercept - H:] = img
    return out


def _brute_force_agrees():
    rng = np.random.default_rng(5)
    img = rng.standard_normal((6, 8))
    P = fr.funnel_ref(img, 10, 12)
    D = oracle.funnel_direct(img, 10, 12)
    return np.allclose(P, D.real, atol=1e-10 * np.abs(D).max())


def _line_lands_on_eq22_23():
    H = W = S = 64
    Hp = 96
    for k, b in [(0.5, 7.0), (-0.375, -12.0)]:
        P = fr.funnel_ref(ridge_image(H, W, Hp, [(k, b)]), S, Hp)
        t, s = np.unravel_index(np.argmax(np.abs(P)), P.shape)
        if abs((s - S // 2) - k * S / 2) > 0.5 or abs((t - Hp // 2) - b) > 1:
            return False
    return True


def test_unmutated_oracle_passes_both_checks():
    assert _brute_force_agrees()
    assert _line_lands_on_eq22_23()


@pytest.mark.parametrize("name,attr,fake", [
    ("step-3 kernel sign", "fourier_xprime", _wrong_sign_step3),
    ("step-1 centring dropped", "fourier_y", _no_centring_step1),
    ("NVMT scale inverted", "nvmt_positions", _inverted_nvmt_positions),
    ("padding all above", "pad_rows", _pad_all_above),
])
def test_planted_mistake_is_caught(monkeypatch, name, attr, fake):
    monkeypatch.setattr(fr, attr, fake)
    assert not (_brute_force_agrees() and _line_lands_on_eq22_23()), name


def test_planted_step4_weight_is_caught(monkeypatch):
    orig = fr.inverse_fourier_omega2

    def halved(G, n_intercept):
        G = G.copy()
        G[1:-1] *= 0.5                          # forgets the factor 2 of the interior bins
        return orig(G, n_intercept)

    monkeypatch.setattr(fr, "inverse_fourier_omega2", halved)
    assert not _brute_force_agrees()
