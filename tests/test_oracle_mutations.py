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


# ------------------------------------------------- line verification (Sec. 4.5)
import inspect                                                     # noqa: E402
import json                                                        # noqa: E402
import os                                                          # noqa: E402

from oracle import verification as vr                              # noqa: E402


def _mutant(old, new):
    """band_profile with one line of its source replaced."""
    src = inspect.getsource(vr.band_profile)
    assert old in src, old
    ns = dict(vr.__dict__)
    exec(src.replace(old, new), ns)
    return ns["band_profile"]


def _verification_pins_hold(band_profile):
    """The closed forms of test_oracle_verify and the Fig. 9 example, for a
    given band_profile."""
    # horizontal ridge on row 11 of a 30-row image in a 64-row frame
    img = np.zeros((30, 48))
    img[11, :] = 2.5
    prof, length = band_profile(img, 11 + 17, 24, 48, 64, 3)
    if not (np.allclose(prof, [0, 0, 0, 2.5, 0, 0, 0]) and length == 48):
        return False
    # step edge: dark rows above, bright from row 16
    img = np.zeros((32, 32))
    img[16:, :] = 0.8
    prof, _ = band_profile(img, 15, 16, 32, 32, 3)
    if not np.allclose(prof, [0, 0, 0, 0, 0.8, 0.8, 0.8]):
        return False
    # linear ramp: p[d] is the mean centre row + d (interpolation and slope)
    img = np.repeat(np.arange(50, dtype=np.float64)[:, None], 40, axis=1)
    prof, _ = band_profile(img, 31, 27, 40, 64, 2)
    slope, offset = vr.band_geometry(31, 27, 40, 64, 50, 40)
    for j, d in enumerate(range(-2, 3)):
        vs = [slope * u + offset + d for u in range(40)]
        vs = [v for v in vs if 0 <= np.floor(v) and np.floor(v) + 1 <= 49]
        if abs(prof[j] - np.mean(vs)) > 1e-9:
            return False
    # a line leaving the image at the bottom: the centre line counts only
    # columns whose two taps are both inside
    img = np.repeat(np.arange(50, dtype=np.float64)[:, None], 40, axis=1)
    t, s = 32 + 13 + 7, 20 + 8                       # k = 0.4, centre row 0.4 (u - 20) + 45
    _, length = band_profile(img, t, s, 40, 64, 1)
    slope, offset = vr.band_geometry(t, s, 40, 64, 50, 40)
    if length != sum(1 for u in range(40) if 0 <= np.floor(slope * u + offset) <= 48):
        return False
    # Fig. 9: the inverse-space peak's line is in the image
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig9_wrapped_peak.json")) as f:
        g = json.load(f)
    W, H = g["width_M"], g["height_N"]
    img = ridge_image(H, W, g["expanded_length"], [(g["slope_k"], float(g["regular_peak_mn"][1]))])
    m_i, n_i = g["inverse_peak_mn"]
    prof, _ = band_profile(img, m_i + (W + H) // 2, n_i + H // 2, H, W + H, 2, inverse=True)
    return vr.contrast(prof) > 0.5 and int(np.argmax(prof)) == 2


def test_unmutated_verification_passes():
    assert _verification_pins_hold(vr.band_profile)


@pytest.mark.parametrize("name,old,new", [
    ("slope sign", "m = s - n_slope // 2", "m = n_slope // 2 - s"),
    ("expansion offset dropped", "top = (n_intercept - H) // 2", "top = 0"),
    ("nearest row instead of interpolation", "f = (num - q * n_slope) / n_slope", "f = 0.0"),
    ("inverse space not transposed", "        a = a.T", "        a = a"),
    ("band offsets reversed", "v0 = q + t - top + d", "v0 = q + t - top - d"),
    ("samples outside the image counted", "if v0 < 0 or v0 + 1 > H - 1:", "if v0 < 0 or v0 > H - 1:"),
])
def test_planted_verification_mistake_is_caught(name, old, new):
    if name == "samples outside the image counted":
        # the mutant reads the row below the image: clamp that tap so it can run
        src = inspect.getsource(vr.band_profile).replace(old, new).replace(
            "sums[j] += (1.0 - f) * a[v0, u] + f * a[v0 + 1, u]",
            "sums[j] += (1.0 - f) * a[v0, u] + f * a[min(v0 + 1, H - 1), u]")
        ns = dict(vr.__dict__)
        exec(src, ns)
        assert not _verification_pins_hold(ns["band_profile"]), name
        return
    assert not _verification_pins_hold(_mutant(old, new)), name


# ------------------------------------------------ Keys' cubic kernel (step 2)
import importlib                                                   # noqa: E402
fd = importlib.import_module("oracle.funnel_direct")
from tests._keys import keys_failures                               # noqa: E402


def _keys_mutant(old, new):
    """keys_cubic with one piece of its source replaced."""
    src = inspect.getsource(fr.keys_cubic)
    assert old in src, old
    ns = dict(fr.__dict__)
    exec(src.replace(old, new), ns)
    return ns["keys_cubic"]


def test_unmutated_keys_kernels_pass():
    assert keys_failures(fr.keys_cubic) == []
    assert keys_failures(np.vectorize(fd._keys)) == []


@pytest.mark.parametrize("name,old,new", [
    ("a = -0.75", "a: float = KEYS_A", "a: float = -0.75"),
    ("8a term typed as 6a", "8.0 * a * s[m2]", "6.0 * a * s[m2]"),
    ("(a + 2) and (a + 3) swapped", "(a + 2.0) * s[m1] ** 3 - (a + 3.0)", "(a + 3.0) * s[m1] ** 3 - (a + 2.0)"),
    ("outer piece sign of 4a", "- 4.0 * a", "+ 4.0 * a"),
    ("outer piece on |s| <= 3", "(s > 1.0) & (s < 2.0)", "(s > 1.0) & (s < 3.0)"),
])
def test_planted_keys_mistake_is_caught(name, old, new):
    assert keys_failures(_keys_mutant(old, new)), name


def test_planted_cubic_tap_order_is_caught(monkeypatch):
    """Weights attached to the wrong taps (k(f) and k(f + 1) exchanged) break the
    Catmull-Rom / quadratic-reproduction pin of step 2."""
    orig = fr.interp_weights

    def swapped(i0, frac, interp):
        taps, w = orig(i0, frac, interp)
        if interp == "cubic":
            w = w[:, [1, 0, 2, 3]]
        return taps, w

    monkeypatch.setattr(fr, "interp_weights", swapped)
    from tests import test_oracle_pins as pins
    with pytest.raises(AssertionError):
        pins.test_cubic_nvmt_row_is_catmull_rom_and_exact_on_quadratics()
