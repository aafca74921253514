"""Seeded synthetic line images for the funnel-transform workloads.

This module only draws pictures: it holds none of the transform's arithmetic and
is shared by the tests, the benchmark and the oracle-side checks.  Every image is
built in float64 from a PCG64 stream seeded with ``SEED_BASE + 1000*workload +
index`` and cast to float32 at the end.

Line model (corner coordinates, row index down, column index right):
``row = k*col + b_c`` with ``k ~ U[-1, 1]`` and ``b_c ~ U[0, H)``.

* ridge line: ``amp * exp(-d^2 / (2 sigma^2))`` with ``d`` the perpendicular
  distance ``|row - k*col - b_c| / sqrt(1 + k^2)``;
* step edge: ``h * [row - k*col - b_c > 0]`` (a half-plane intensity step);
* occluder: per line a fraction ``f ~ U[0, occlusion_max]`` of its in-image
  extent is covered by a rectangle (the sub-segment's bounding box dilated by
  ``3 sigma`` for ridges, 2 px for steps) painted with the background level;
* noise: additive ``N(0, noise_sigma^2)`` after painting.

The background level of an image is one draw of ``N(0.2, 0.05^2)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

SEED_BASE = 190409409

# Workload identifiers (the number used in the seed).
WL_SINGLE_256 = 1      # one 256x256 image, 3 ridges
WL_BATCH_1024 = 2      # 64 x 1024^2, mixed content
WL_VARLEN = 3          # 512 mixed-size images
WL_GRAD_512 = 4        # 32 x 512^2
WL_LARGE_4096 = 5      # 8 x 4096^2, 100 lines
VARLEN_SIDES = (128, 192, 256, 384, 512, 768, 1024, 1536, 2048)


@dataclass
class Line:
    kind: str          # "ridge" or "step"
    k: float           # slope in corner coordinates
    b_c: float         # row at column 0
    sigma: float       # ridge width in px (0 for steps)
    amp: float         # ridge amplitude or step height


@dataclass
class SynthImage:
    img: np.ndarray                  # (H, W) float32
    lines: List[Line] = field(default_factory=list)
    background: float = 0.0
    noise_sigma: float = 0.0


def rng_for(workload: int, index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * workload + index))


def render_ridge(img: np.ndarray, k: float, b_c: float, sigma: float, amp: float) -> None:
    """Add a Gaussian-profile ridge; evaluated in a band of +-6 sigma around the line."""
    H, W = img.shape
    s = np.sqrt(1.0 + k * k)
    reach = int(np.ceil(6.0 * sigma * s)) + 1
    cols = np.arange(W)
    centre = k * cols + b_c
    base = np.floor(centre).astype(np.int64)
    offs = np.arange(-reach, reach + 2)
    rows = base[:, None] + offs[None, :]                      # (W, band)
    ok = (rows >= 0) & (rows < H)
    d = (rows - centre[:, None]) / s
    val = amp * np.exp(-(d * d) / (2.0 * sigma * sigma))
    cc = np.broadcast_to(cols[:, None], rows.shape)
    img[rows[ok], cc[ok]] += val[ok]


def render_step(img: np.ndarray, k: float, b_c: float, h: float) -> None:
    H, W = img.shape
    rows = np.arange(H)[:, None]
    thr = (k * np.arange(W) + b_c)[None, :]
    img += h * (rows > thr)


def step_first_rows(H: int, W: int, k: float, b_c: float) -> np.ndarray:
    """Per column, the first row strictly below the edge row = k*col + b_c
    (H where there is none): the rows that render_step raises start there."""
    thr = k * np.arange(W) + b_c
    return np.clip(np.floor(thr).astype(np.int64) + 1, 0, H)


def line_col_extent(H: int, W: int, k: float, b_c: float) -> Tuple[float, float]:
    """Column interval over which row = k*col + b_c stays inside [0, H-1]."""
    lo, hi = 0.0, float(W - 1)
    if k > 0:
        hi = min(hi, (H - 1 - b_c) / k)
        lo = max(lo, (0.0 - b_c) / k)
    elif k < 0:
        hi = min(hi, (0.0 - b_c) / k)
        lo = max(lo, (H - 1 - b_c) / k)
    return lo, max(lo, hi)


def occlude(img: np.ndarray, line: Line, frac: float, rng: np.random.Generator,
            background: float) -> None:
    H, W = img.shape
    lo, hi = line_col_extent(H, W, line.k, line.b_c)
    span = (hi - lo) * frac
    if span <= 0.0:
        return
    c0 = lo + rng.uniform(0.0, max(hi - lo - span, 0.0))
    c1 = c0 + span
    r0, r1 = sorted((line.k * c0 + line.b_c, line.k * c1 + line.b_c))
    pad = 3.0 * line.sigma if line.kind == "ridge" else 2.0
    ca, cb = int(np.floor(c0 - pad)), int(np.ceil(c1 + pad))
    ra, rb = int(np.floor(r0 - pad)), int(np.ceil(r1 + pad))
    img[max(ra, 0):min(rb + 1, H), max(ca, 0):min(cb + 1, W)] = background


def draw_lines(rng: np.random.Generator, n_lines: int, H: int, ridge_frac: float,
               ridge_sigma: Tuple[float, float], ridge_amp: float,
               step_h: Tuple[float, float]) -> List[Line]:
    lines = []
    for _ in range(n_lines):
        k = rng.uniform(-1.0, 1.0)
        b_c = rng.uniform(0.0, H)
        if rng.uniform() < ridge_frac:
            sig = rng.uniform(*ridge_sigma) if ridge_sigma[0] != ridge_sigma[1] else ridge_sigma[0]
            lines.append(Line("ridge", k, b_c, sig, ridge_amp))
        else:
            lines.append(Line("step", k, b_c, 0.0, rng.uniform(*step_h)))
    return lines


def compose(rng: np.random.Generator, H: int, W: int, lines: Sequence[Line],
            occlusion_max: float, noise_sigma: float, background: float) -> SynthImage:
    img = np.full((H, W), background, dtype=np.float64)
    steps = np.zeros((H + 1, W), dtype=np.float64)      # step heights at their first rows
    cols = np.arange(W)
    for ln in lines:
        if ln.kind == "ridge":
            render_ridge(img, ln.k, ln.b_c, ln.sigma, ln.amp)
        else:
            steps[step_first_rows(H, W, ln.k, ln.b_c), cols] += ln.amp
    if any(ln.kind == "step" for ln in lines):
        img += np.cumsum(steps, axis=0)[:H]              # the same half-planes as render_step
    if occlusion_max > 0.0:
        for ln in lines:
            occlude(img, ln, rng.uniform(0.0, occlusion_max), rng, background)
    if noise_sigma > 0.0:
        img += rng.normal(0.0, noise_sigma, size=img.shape)
    return SynthImage(img.astype(np.float32), list(lines), background, noise_sigma)


def single_256(index: int = 0) -> SynthImage:
    """256x256, background N(0.2, 0.05^2), 3 ridges (sigma 1.5 px, amp 1), noise 0.1."""
    rng = rng_for(WL_SINGLE_256, index)
    bg = rng.normal(0.2, 0.05)
    lines = draw_lines(rng, 3, 256, 1.0, (1.5, 1.5), 1.0, (0.0, 0.0))
    return compose(rng, 256, 256, lines, 0.0, 0.1, bg)


def mixed_image(workload: int, index: int, H: int, W: int,
                n_lines: int | None = None, noise_sigma: float | None = None) -> SynthImage:
    """1-20 lines (or ``n_lines``), 50/50 ridge (sigma U[1,3]) / step (h U[0.3,1]),
    occluders over 0-30% of each line, noise sigma U[0.05, 0.5] (or fixed)."""
    rng = rng_for(workload, index)
    bg = rng.normal(0.2, 0.05)
    n = int(rng.integers(1, 21)) if n_lines is None else int(n_lines)
    lines = draw_lines(rng, n, H, 0.5, (1.0, 3.0), 1.0, (0.3, 1.0))
    ns = rng.uniform(0.05, 0.5) if noise_sigma is None else float(noise_sigma)
    return compose(rng, H, W, lines, 0.30, ns, bg)


def batch_1024(count: int = 64, start: int = 0, side: int = 1024) -> np.ndarray:
    """``count`` mixed-content images of ``side`` x ``side`` as one (count, side, side) array."""
    out = np.empty((count, side, side), dtype=np.float32)
    for i in range(count):
        out[i] = mixed_image(WL_BATCH_1024, start + i, side, side).img
    return out


def grad_batch_512(count: int = 32, start: int = 0, side: int = 512) -> List[SynthImage]:
    return [mixed_image(WL_GRAD_512, start + i, side, side) for i in range(count)]


def large_4096(count: int = 8, start: int = 0, side: int = 4096) -> List[SynthImage]:
    return [mixed_image(WL_LARGE_4096, start + i, side, side, n_lines=100, noise_sigma=0.2)
            for i in range(count)]


def varlen_shapes(count: int = 512) -> List[Tuple[int, int]]:
    rng = rng_for(WL_VARLEN, 999_999)
    sides = np.asarray(VARLEN_SIDES)
    return [(int(sides[rng.integers(len(sides))]), int(sides[rng.integers(len(sides))]))
            for _ in range(count)]


def varlen_image(index: int, H: int, W: int) -> SynthImage:
    return mixed_image(WL_VARLEN, index, H, W)


def blob_target(n_intercept: int, n_slope: int, cells, sigma: float = 2.0, amp: float = 1.0) -> np.ndarray:
    """Target map of the gradient workload: Gaussian blobs (sigma in cells,
    periodic in both axes) centred at the given (t, s) cells, summed."""
    t = np.arange(n_intercept)[:, None]
    s = np.arange(n_slope)[None, :]
    out = np.zeros((n_intercept, n_slope), dtype=np.float64)
    for (tc, sc) in cells:
        dt = (t - tc + n_intercept / 2.0) % n_intercept - n_intercept / 2.0
        ds = (s - sc + n_slope / 2.0) % n_slope - n_slope / 2.0
        out += amp * np.exp(-(dt * dt + ds * ds) / (2.0 * sigma * sigma))
    return out.astype(np.float32)
