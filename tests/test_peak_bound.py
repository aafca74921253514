"""The argument behind peak detection from tile maxima, checked on the CPU.

The detected list of Sec. 4.4 is the top K strict local maxima of the order
(|P| descending, linear index ascending).  A peak never exceeds the maximum M of
its tile, so once K peaks are known, a tile whose M is below the K-th of them
cannot contribute.  This file replays the procedure of the peak pass in plain
NumPy: round 1 takes every valid tile whose maximum reaches T, the nw-th largest
valid maximum (ties included); tiles run nw per batch; in a batch every tile
marks its strict local maxima at or above the bound and reports its best marked
value, the K-th largest of those (K <= nw) cuts the appends, the candidates are
cut back to the best K, which raises the bound; round 2 takes every other valid
tile whose maximum reaches the bound.  It must reproduce the oracle's list
procedure exactly, on maps built to stress it: ties, plateaus across tile
borders, tile maxima on borders next to brighter cells, thresholds, ragged last
tiles and K above the number of peaks; mistakes planted in the replay (no second
round, strict comparisons, an off-by-one cut) must change some list.  The CUDA
kernel is checked against the oracle by the GPU tests; this pins the procedure.
"""
import numpy as np
import pytest

import oracle


def strict_local_maxima(A):
    """Boolean map: cell precedes all 8 (wrapped) neighbours in the order."""
    Hp, S = A.shape
    idx = np.arange(Hp * S).reshape(Hp, S)
    ok = np.ones(A.shape, dtype=bool)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            if a == 0 and b == 0:
                continue
            nv = np.roll(np.roll(A, -a, 0), -b, 1)
            ni = np.roll(np.roll(idx, -a, 0), -b, 1)
            ok &= ~((nv > A) | ((nv == A) & (ni < idx)))
    return ok


def tile_bound_peaks(A, K, thr, th, tw, warps, round2=True, strict=False, cut_strict=False, cut_rank=0):
    """Peaks read from the tiles that the bound admits; returns (list, tiles read).
    The keyword arguments plant mistakes: round2=False drops the second round,
    strict=True admits a tile only when its maximum exceeds the bound, cut_strict
    appends only cells strictly above the cut, cut_rank=-1 takes the cut from
    the (K-1)-th best tile value instead of the K-th."""
    Hp, S = A.shape
    lm = strict_local_maxima(A)
    nty, ntx = -(-Hp // th), -(-S // tw)
    M = np.array([[A[ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw].max() for tx in range(ntx)]
                  for ty in range(nty)]).ravel()
    state = {"cand": [], "bound": thr, "read": 0}

    def marks(tile, bound):
        ty, tx = divmod(tile, ntx)
        state["read"] += 1
        return [(float(A[t, s]), t * S + s)
                for t in range(ty * th, min((ty + 1) * th, Hp))
                for s in range(tx * tw, min((tx + 1) * tw, S))
                if A[t, s] >= bound and lm[t, s]]

    def run(tiles):
        for b0 in range(0, len(tiles), warps):
            bound = state["bound"]
            marked = [marks(tile, bound) for tile in tiles[b0:b0 + warps]
                      if M[tile] > bound or (M[tile] == bound and not strict)]
            cut = bound
            bests = sorted((max(v for v, _ in mk) for mk in marked if mk), reverse=True)
            r = K - 1 + cut_rank
            if K <= warps and 0 <= r < len(bests) and len(bests) >= K:
                cut = max(cut, bests[r])
            for mk in marked:
                state["cand"] += [(-v, lin) for v, lin in mk if (v > cut if cut_strict else v >= cut)]
            if len(state["cand"]) >= K:          # keep the best K, raise the bound
                state["cand"] = sorted(state["cand"])[:K]
                state["bound"] = max(state["bound"], -state["cand"][-1][0])

    valid = [i for i in range(M.size) if M[i] >= thr]
    top = sorted((M[i] for i in valid), reverse=True)
    T = top[warps - 1] if len(top) >= warps else -np.inf
    run([i for i in valid if M[i] >= T])
    if round2:
        run([i for i in valid if M[i] < T and M[i] >= state["bound"]])
    out = sorted(state["cand"])[:K]
    return [(lin // S, lin % S, -v) for v, lin in out], state["read"]


def maps(kind, rng, Hp, S):
    if kind == "noise":
        return rng.standard_normal((Hp, S))
    if kind == "ties":
        return rng.integers(-3, 4, size=(Hp, S)).astype(np.float64)
    if kind == "plateaus":
        b = rng.integers(0, 5, size=(Hp // 5 + 1, S // 5 + 1)).astype(np.float64)
        return np.kron(b, np.ones((5, 5)))[:Hp, :S]
    if kind == "border_max":
        m = rng.uniform(0.0, 1.0, size=(Hp, S))
        for t0 in range(0, Hp, 8):
            for s0 in range(0, S, 8):
                if t0 + 7 < Hp and s0 + 3 < S:
                    m[t0 + 7, s0 + 3] = 50.0 + t0 + s0 / 100.0
                    m[(t0 + 8) % Hp, s0 + 3] = 60.0 + t0 + s0 / 100.0
        return m
    if kind == "peaks":                          # a few bright peaks over noise
        m = 0.1 * rng.standard_normal((Hp, S))
        for _ in range(6):
            m[rng.integers(Hp), rng.integers(S)] += rng.uniform(5, 10)
        return m
    return np.zeros((Hp, S))


@pytest.mark.parametrize("kind", ["noise", "ties", "plateaus", "border_max", "peaks", "zero"])
@pytest.mark.parametrize("Hp,S,th,tw", [(32, 48, 8, 8), (40, 36, 8, 16), (24, 30, 4, 8), (6, 10, 4, 4)])
@pytest.mark.parametrize("K", [1, 3, 17, 400])
def test_tile_bound_reproduces_the_list_procedure(kind, Hp, S, th, tw, K):
    rng = np.random.default_rng(Hp * 1000 + S + K)
    A = np.abs(maps(kind, rng, Hp, S))
    for thr in (-np.inf, 0.5):
        got, _ = tile_bound_peaks(A, K, thr, th, tw, warps=4)
        assert got == oracle.peaks_ref(A, K, thr), (kind, thr)


def test_tile_bound_reads_few_tiles_when_peaks_stand_out():
    """With a few bright peaks and top_k = 3 the bound admits only the tiles of
    those peaks after the first batch: most tiles are never read."""
    rng = np.random.default_rng(7)
    A = np.abs(maps("peaks", rng, 64, 64))
    got, read = tile_bound_peaks(A, 3, -np.inf, 8, 8, warps=4)
    assert got == oracle.peaks_ref(A, 3)
    assert read <= 8                                   # of 64 tiles


@pytest.mark.parametrize("mistake", [{"round2": False}, {"strict": True}, {"cut_strict": True}, {"cut_rank": -1}])
def test_planted_mistakes_are_caught(mistake):
    """Dropping the second round, admitting a tile only when its maximum is
    strictly above the bound, appending only cells strictly above the cut, or
    taking the cut from the (K-1)-th best tile value changes the list on some of
    the maps above."""
    caught = False
    for kind in ("noise", "ties", "plateaus", "border_max", "peaks"):
        for Hp, S, th, tw in ((32, 48, 8, 8), (24, 30, 4, 8)):
            for K in (3, 17):
                rng = np.random.default_rng(Hp * 1000 + S + K)
                A = np.abs(maps(kind, rng, Hp, S))
                got, _ = tile_bound_peaks(A, K, -np.inf, th, tw, warps=4, **mistake)
                caught |= got != oracle.peaks_ref(A, K)
    assert caught
