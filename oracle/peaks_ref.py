"""List-based peak detection of Sec. 4.4 and the peak-to-line maps of Sec. 4.3.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 4.4: every cell of the parameter space is put in a candidate list sorted
by brightness, descending.  Cells are visited in that order; a visited cell is
accepted as a peak unless a cell of its 3 x 3 neighbourhood was visited before
it, and is marked visited either way.  Visiting stops once the detected list
holds the requested number of peaks, or at the first visited cell whose
brightness is below the threshold T.

Readings: equal brightness is ordered by the row-major linear index t*S + s
(ascending); the neighbourhood wraps around both axes (the map is periodic in
slope and intercept, eqs. 20-21); brightness is |P| (Sec. 3.3).
"""
from __future__ import annotations

import numpy as np


def peaks_ref(A: np.ndarray, top_k: int, threshold: float = -np.inf):
    """Returns a list of (t, s, value) in detection order for the brightness map
    A[t, s] (t: intercept row, s: slope column)."""
    A = np.asarray(A)
    Hp, S = A.shape
    flat = A.ravel()
    order = np.lexsort((np.arange(flat.size), -flat))   # brightness desc, index asc
    visited = np.zeros((Hp, S), dtype=bool)
    found = []
    if top_k <= 0:
        return found
    for p in order:
        p = int(p)
        v = flat[p]
        if v < threshold:
            break
        t, s = divmod(p, S)
        rows = [(t - 1) % Hp, t, (t + 1) % Hp]
        cols = [(s - 1) % S, s, (s + 1) % S]
        seen = visited[np.ix_(rows, cols)].any()
        visited[t, s] = True
        if not seen:
            found.append((t, s, float(v)))
            if len(found) == top_k:
                break
    return found


def peak_to_line(t: int, s: int, n_slope: int, n_intercept: int):
    """Regular space, eqs. (22)-(23): m = s - S/2, n = t - H'/2, k = 2 m / S, b_y = n
    (centred coordinates of the expanded image)."""
    m = s - n_slope // 2
    n = t - n_intercept // 2
    return 2.0 * m / n_slope, float(n)


def inverse_peak_to_line(t: int, s: int, n_inv_slope: int, n_x_intercept: int):
    """Inverse space, eqs. (24)-(25): 1/k = 2 n / N, b_x = m, with the inverse map
    stored as Q[t, s], t = b_x + W'/2 and s = n + N/2."""
    n = s - n_inv_slope // 2
    m = t - n_x_intercept // 2
    return 2.0 * n / n_inv_slope, float(m)
