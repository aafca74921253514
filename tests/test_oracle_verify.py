"""Pins of the line-verification oracle (Sec. 4.5) against closed forms and
the paper's worked example (Fig. 9): the wrapping peak's line does not exist,
the inverse-space peak's line does."""
import json
import os

import numpy as np

from oracle import verification as vr
from tests._lines import ridge_image

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_constant_image_has_flat_profile_and_no_line():
    img = np.full((40, 64), 0.7)
    # k = 0 (s = S/2), centre row 20 of the 40-row image inside the 64-row frame (top = 12)
    prof, length = vr.band_profile(img, 32 + (20 + 12 - 32), 32, 64, 64, 2)
    assert np.allclose(prof, 0.7) and length == 64
    assert vr.contrast(prof) < 1e-12
    assert not vr.verify_ref(img, [(32, 32)], 64, 64, 2, 0.05, 10)[0][2]


def test_horizontal_ridge_closed_form():
    H, W, Hp, S = 30, 48, 64, 48
    top = (Hp - H) // 2
    img = np.zeros((H, W))
    img[11, :] = 2.5
    t = 11 + top                       # n = t - Hp/2 = row + top - Hp/2: the line y = n through row 11
    prof, length = vr.band_profile(img, t, S // 2, S, Hp, 3)
    assert np.allclose(prof, [0, 0, 0, 2.5, 0, 0, 0]) and length == W
    assert abs(vr.contrast(prof) - 2.5) < 1e-12


def test_linear_ramp_profile_is_the_mean_centre_plus_offset():
    """Linear interpolation along the band: on I[row, col] = row every sample is
    its own row coordinate, so p[d] = mean over valid columns of v_c(u) + d."""
    H, W, Hp, S = 50, 40, 64, 40
    img = np.repeat(np.arange(H, dtype=np.float64)[:, None], W, axis=1)
    t, s = 31, 27                      # k = 2 * 7 / 40 = 0.35, n = -1
    slope, offset = vr.band_geometry(t, s, S, Hp, H, W)
    assert abs(slope - 0.35) < 1e-15
    prof, length = vr.band_profile(img, t, s, S, Hp, 2)
    for j, d in enumerate(range(-2, 3)):
        vs = [slope * u + offset + d for u in range(W)]
        vs = [v for v in vs if 0 <= np.floor(v) and np.floor(v) + 1 <= H - 1]
        assert abs(prof[j] - np.mean(vs)) < 1e-9
    assert length == sum(1 for u in range(W) if 0 <= np.floor(slope * u + offset) <= H - 2)


def test_step_edge_contrast():
    H, W, Hp, S = 32, 32, 32, 32
    img = np.zeros((H, W))
    img[16:, :] = 0.8                  # rows 16.. bright: an edge between rows 15 and 16
    prof, _ = vr.band_profile(img, 15, 16, S, Hp, 3)   # centre line on row 15 (top = 0)
    assert np.allclose(prof, [0, 0, 0, 0, 0.8, 0.8, 0.8])
    assert abs(vr.contrast(prof) - 0.4) < 1e-12


def test_fig9_wrapping_peak_is_rejected_and_inverse_peak_verified():
    with open(os.path.join(GOLDEN, "fig9_wrapped_peak.json")) as f:
        g = json.load(f)
    W, H, k = g["width_M"], g["height_N"], g["slope_k"]
    Hp = g["expanded_length"]
    img = ridge_image(H, W, Hp, [(k, float(g["regular_peak_mn"][1]))], sigma=1.0, amp=1.0)
    m_r, n_r = g["regular_peak_mn"]
    (prof_r, len_r, ok_r), = vr.verify_ref(img, [(n_r + Hp // 2, m_r + W // 2)], W, Hp, 2, 0.2, 20)
    m_i, n_i = g["inverse_peak_mn"]
    (prof_i, len_i, ok_i), = vr.verify_ref(img, [(m_i + (W + H) // 2, n_i + H // 2)], H, W + H, 2, 0.2, 20,
                                          inverse=True)
    assert not ok_r and vr.contrast(prof_r) < 0.05       # the line of slope -0.73 is not in the image
    assert ok_i and vr.contrast(prof_i) > 0.5            # the line of slope 3.27 is
    assert int(np.argmax(prof_i)) == 2 and len_i > 300   # centred on the band, along most of the rows


def test_line_leaving_the_image_counts_inside_samples_only():
    """Centre row 0.4 (u - 20) + 45 of a 50-row image (in a 64-row frame, top 7):
    it leaves the image at the bottom, and only columns whose two taps are both
    inside count."""
    H, W, Hp, S = 50, 40, 64, 40
    img = np.repeat(np.arange(H, dtype=np.float64)[:, None], W, axis=1)
    t, s = 32 + 13 + 7, 20 + 8
    slope, offset = vr.band_geometry(t, s, S, Hp, H, W)
    assert abs(slope - 0.4) < 1e-15 and abs(offset - 37.0) < 1e-12
    prof, length = vr.band_profile(img, t, s, S, Hp, 1)
    inside = [u for u in range(W) if 0 <= np.floor(slope * u + offset) <= H - 2]
    assert length == len(inside) and 0 < length < W
    assert abs(prof[1] - np.mean([slope * u + offset for u in inside])) < 1e-9
