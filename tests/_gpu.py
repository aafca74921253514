"""Helpers shared by the GPU parity tests (device memory through torch, every
compute step through the C ABI)."""
import os

import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_09409_gb300 import funnel as f
    if not os.path.exists(f.LIB_PATH):
        from paper_1904_09409_gb300 import build
        build.build()
    f.lib()
    return torch


def forward(plan, imgs):
    """imgs: (B, H, W) float32 numpy -> (B, H', S) float32 numpy via ft_forward."""
    import torch
    from paper_1904_09409_gb300 import funnel as f
    x = torch.from_numpy(np.ascontiguousarray(imgs, dtype=np.float32)).cuda()
    m = torch.full((x.shape[0], plan.Hp, plan.S), float("nan"), dtype=torch.float32, device="cuda")
    f.ft_forward(plan, x, m)
    torch.cuda.synchronize()
    return m.cpu().numpy()


def backward(plan, grads):
    import torch
    from paper_1904_09409_gb300 import funnel as f
    g = torch.from_numpy(np.ascontiguousarray(grads, dtype=np.float32)).cuda()
    gi = torch.full((g.shape[0], plan.H, plan.W), float("nan"), dtype=torch.float32, device="cuda")
    f.ft_backward(plan, g, gi)
    torch.cuda.synchronize()
    return gi.cpu().numpy()


def peaks(plan, maps, top_k, threshold=float("-inf")):
    """maps: (B, H', S) float32 numpy -> list of [(t, s, value)] via ft_peaks."""
    import torch
    from paper_1904_09409_gb300 import funnel as f
    m = torch.from_numpy(np.ascontiguousarray(maps, dtype=np.float32)).cuda()
    out, cnt = f.ft_peaks(plan, m, top_k, threshold)
    torch.cuda.synchronize()
    res = f.peaks_to_numpy(out, cnt, top_k)
    return [[(int(p["t"]), int(p["s"]), float(p["value"])) for p in r] for r in res], res


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def robust_rank_mismatches(ref_map, ref_peaks, got_peaks, tol):
    """Ranks i where the FP64 list is unambiguous (its local-max margin and the
    brightness gaps to ranks i-1 and i+1 all exceed tol) but the GPU list differs."""
    A = np.abs(ref_map)
    Hp, S = A.shape
    bad = []
    vals = [v for _, _, v in ref_peaks]
    for i, (t, s, v) in enumerate(ref_peaks):
        nb = max(A[(t + dt) % Hp, (s + ds) % S] for dt in (-1, 0, 1) for ds in (-1, 0, 1)
                 if (dt, ds) != (0, 0))
        if v - nb <= tol:
            continue
        if i > 0 and vals[i - 1] - v <= tol:
            continue
        if i + 1 < len(vals) and v - vals[i + 1] <= tol:
            continue
        if i >= len(got_peaks) or got_peaks[i][:2] != (t, s):
            bad.append((i, (t, s), got_peaks[i][:2] if i < len(got_peaks) else None))
    return bad
