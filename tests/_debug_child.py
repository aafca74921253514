"""Child process of tests/test_gpu_debug.py: loads the bounds-checked build
(FT_DEBUG=1 before the binding is imported), runs the transform, its adjoint and
both peak passes on small and odd-radix sizes, compares with the FP64 oracle and
prints OK when every result matches and no device index check fired."""
import os
import sys

import numpy as np

os.environ["FT_DEBUG"] = "1"
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch                                            # noqa: E402

import oracle                                           # noqa: E402
from paper_1904_09409_gb300 import funnel as f          # noqa: E402

assert f.LIB_PATH.endswith("libfunnel_debug.so"), f.LIB_PATH
assert f.ft_debug_build()
assert f.ft_debug_flags() == 0

# (H, W, S, H'): the fixed-length kernels start at 128 (and 192); the others
# run the generic kernels (radix 2 / 3 / 4 / 8 mixes), all with the checks
CASES = [(8, 8, 8, 8), (16, 16, 16, 16), (32, 32, 32, 32), (64, 64, 64, 64), (6, 4, 6, 6), (12, 18, 18, 24),
         (24, 36, 36, 54), (48, 54, 72, 96), (20, 30, 36, 48), (128, 128, 128, 128), (100, 96, 192, 192),
         (192, 192, 192, 192), (256, 128, 128, 256)]
rng = np.random.default_rng(9)
bad = []
for H, W, S, Hp in CASES:
    for interp in ("linear", "cubic"):
        x = rng.standard_normal((2, H, W)).astype(np.float32)
        g = rng.standard_normal((2, Hp, S)).astype(np.float32)
        with f.Plan(H, W, S, Hp, interp) as plan:
            xd = torch.from_numpy(x).cuda()
            m = torch.empty((2, Hp, S), device="cuda")
            f.ft_forward(plan, xd, m)
            gi = torch.empty((2, H, W), device="cuda")
            f.ft_backward(plan, torch.from_numpy(g).cuda(), gi)
            K = min(8, Hp * S // 4)
            out, cnt = f.ft_peaks(plan, m, K)
            m2 = torch.empty_like(m)
            out2, cnt2 = f.ft_detect(plan, xd, m2, K)
            torch.cuda.synchronize()
            maps, grads = m.cpu().numpy(), gi.cpu().numpy()
            pk = f.peaks_to_numpy(out, cnt, K)
            pk2 = f.peaks_to_numpy(out2, cnt2, K)
        for i in range(2):
            ref = oracle.funnel_ref(x[i], S, Hp, interp)
            e = np.linalg.norm(maps[i] - ref) / np.linalg.norm(ref)
            eg = np.linalg.norm(grads[i] - oracle.adjoint_ref(g[i].astype(np.float64), H, W, interp))
            eg /= np.linalg.norm(oracle.adjoint_ref(g[i].astype(np.float64), H, W, interp))
            want = [(t, s) for t, s, _ in oracle.peaks_ref(np.abs(maps[i]).astype(np.float64), K)]
            got = [(int(p["t"]), int(p["s"])) for p in pk[i]]
            got2 = [(int(p["t"]), int(p["s"])) for p in pk2[i]]
            if e > 1e-5 or eg > 1e-5 or got != want or got2 != want:
                bad.append((H, W, S, Hp, interp, i, e, eg))
flags = f.ft_debug_flags()
print("flags", flags, "mismatches", bad)
print("OK" if flags == 0 and not bad else "FAIL")
