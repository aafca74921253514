"""Test helpers: place lines given in the paper's centred coordinates.

Centred coordinates of an image expanded to n_intercept rows (Sec. 4.2):
x = col - W/2, y = row + top - H'/2 with top = (H' - H)//2 zero rows above.
A line y = k x + b therefore has row = k*col + b_c in the image's own corner
coordinates with b_c = b - k W/2 + H'/2 - top.
"""
import numpy as np

from paper_1904_09409_gb300 import synth


def corner_intercept(k, b, H, W, n_intercept):
    top = (n_intercept - H) // 2
    return b - k * W / 2.0 + n_intercept / 2.0 - top


def centred_intercept(k, b_c, H, W, n_intercept):
    top = (n_intercept - H) // 2
    return b_c + k * W / 2.0 - n_intercept / 2.0 + top


def ridge_image(H, W, n_intercept, lines, sigma=1.0, amp=1.0):
    """lines: iterable of (k, b) in centred coordinates."""
    img = np.zeros((H, W))
    for k, b in lines:
        synth.render_ridge(img, k, corner_intercept(k, b, H, W, n_intercept), sigma, amp)
    return img


def wrap_centred(v, period):
    """Wrap v into [-period/2, period/2)."""
    return (v + period / 2.0) % period - period / 2.0


def true_cells(lines, H, W, n_slope, n_intercept):
    """Map cells (t, s) where the drawn lines should peak: eqs. (22)-(23) with the
    corner-to-centred conversion, slope and intercept wrapped into the map."""
    cells = []
    for ln in lines:
        b = centred_intercept(ln.k, ln.b_c, H, W, n_intercept)
        t = (b + n_intercept / 2.0) % n_intercept
        s = (ln.k * n_slope / 2.0 + n_slope / 2.0) % n_slope
        cells.append((t, s))
    return cells
