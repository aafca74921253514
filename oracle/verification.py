"""Line verification of Sec. 4.5 (post-processing of the detected list).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 4.5 verifies every peak of the detected list: the peak's coordinates give
a candidate line (eqs. 22-23 in the regular space, 24-25 in the inverse space);
a band of 3 to 7 pixels centred on that line is cut from the original image
and integrated along the line's length, which leaves a one-dimensional profile
across the band; the profile tells whether the line exists, and a peak whose
line does not exist (a wrapping peak, a false peak) leaves the list.

Readings (the paper fixes the steps, not the numbers):

* Band geometry.  A regular-space peak at map cell (t, s) of an n_intercept x
  n_slope map gives m = s - S/2, n = t - H'/2 and the line y = (2m/S) x + n in
  the centred coordinates of the expanded image, x = col - W/2,
  y = row + top - H'/2, top = (H' - H) // 2.  Its band runs along the columns:
  for every column u the centre row is v_c(u) = (2m/S)(u - W/2) + n + H'/2 - top
  and the band samples rows v_c(u) + d, d = -h .. h (width 2h + 1), by linear
  interpolation between the two nearest rows.  A sample counts only where both
  rows lie inside the image.  An inverse-space peak is the regular-space peak of
  the transposed image (eqs. 24-25), so the same geometry applies with rows and
  columns exchanged.
* Integration.  profile[d] = the mean of the valid samples at offset d along the
  band; length = the number of valid samples on the centre line.
* Decision (step 4).  contrast = max(|p[0] - (p[-h] + p[h]) / 2|,
  |p[h] - p[-h]| / 2): a ridge raises the centre over both borders, a step edge
  separates the two borders.  The line exists iff length >= min_length and
  contrast >= min_contrast.
"""
from __future__ import annotations

import numpy as np


def band_geometry(t: int, s: int, n_slope: int, n_intercept: int, H: int, W: int):
    """(slope, offset) of v_c(u) = slope * u + offset for the regular-space cell
    (t, s) of an image with H rows and W columns expanded to n_intercept rows."""
    m = s - n_slope // 2
    n = t - n_intercept // 2
    top = (n_intercept - H) // 2
    k = 2.0 * m / n_slope
    return k, -k * W / 2.0 + n + n_intercept / 2.0 - top


def band_profile(img: np.ndarray, t: int, s: int, n_slope: int, n_intercept: int, half_width: int,
                 inverse: bool = False):
    """Mean band profile p[d], d = -h .. h, and the centre-line length of the
    candidate line of map cell (t, s).  For an inverse-space peak pass the
    original image and inverse=True (the band then runs along the rows)."""
    a = np.asarray(img, dtype=np.float64)
    if inverse:
        a = a.T
    H, W = a.shape
    m = s - n_slope // 2
    top = (n_intercept - H) // 2
    h = half_width
    sums = np.zeros(2 * h + 1)
    counts = np.zeros(2 * h + 1, dtype=np.int64)
    for u in range(W):
        # v_c(u) = (2m/S)(u - W/2) + n + H'/2 - top = m (2u - W) / S + t - top,
        # split exactly into an integer floor and a fraction
        num = m * (2 * u - W)
        q = num // n_slope
        f = (num - q * n_slope) / n_slope
        for j, d in enumerate(range(-h, h + 1)):
            v0 = q + t - top + d
            if v0 < 0 or v0 + 1 > H - 1:
                continue
            sums[j] += (1.0 - f) * a[v0, u] + f * a[v0 + 1, u]
            counts[j] += 1
    prof = np.where(counts > 0, sums / np.maximum(counts, 1), 0.0)
    return prof, int(counts[h])


def contrast(prof: np.ndarray) -> float:
    h = (len(prof) - 1) // 2
    ridge = abs(prof[h] - 0.5 * (prof[0] + prof[2 * h]))
    step = 0.5 * abs(prof[2 * h] - prof[0])
    return float(max(ridge, step))


def verify_ref(img: np.ndarray, peaks, n_slope: int, n_intercept: int, half_width: int,
               min_contrast: float, min_length: int, inverse: bool = False):
    """[(profile, length, exists)] for the (t, s) cells in ``peaks``."""
    out = []
    for (t, s) in peaks:
        prof, length = band_profile(img, t, s, n_slope, n_intercept, half_width, inverse)
        out.append((prof, length, bool(length >= min_length and contrast(prof) >= min_contrast)))
    return out
