"""Child process of tests/test_zz_no_alloc.py: ft_peaks_noalloc before and after
cudaDeviceReset (which destroys the context that held the scratch array's
address), with device memory from the CUDA runtime directly (no torch, whose
allocator would not survive the reset).  Prints OK when both calls agree with
the oracle's list procedure on the same FP32 maps."""
import ctypes
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle                                            # noqa: E402
from paper_1904_09409_gb300 import funnel as f          # noqa: E402

L = f.lib()
RT = ctypes.CDLL("libcudart.so.13")                     # the runtime libfunnel.so uses
vp, sz = ctypes.c_void_p, ctypes.c_size_t


def check(e, what):
    if e != 0:
        raise SystemExit(f"{what}: CUDA error {e}")


def detect(maps, K):
    batch, Hp, S = maps.shape
    dm, do, dc = vp(), vp(), vp()
    check(RT.cudaMalloc(ctypes.byref(dm), sz(maps.nbytes)), "cudaMalloc")
    check(RT.cudaMalloc(ctypes.byref(do), sz(batch * K * f.PEAK_DTYPE.itemsize)), "cudaMalloc")
    check(RT.cudaMalloc(ctypes.byref(dc), sz(batch * 4)), "cudaMalloc")
    check(RT.cudaMemcpy(dm, maps.ctypes.data_as(vp), sz(maps.nbytes), 1), "cudaMemcpy")
    st = L.ft_peaks_noalloc(dm, Hp, S, batch, K, ctypes.c_float(float("-inf")), do, dc, None)
    if st != f.FT_OK:
        raise SystemExit(f"ft_peaks_noalloc: status {st} ({L.ft_last_error().decode()})")
    check(RT.cudaDeviceSynchronize(), "cudaDeviceSynchronize")
    out = np.zeros(batch * K, f.PEAK_DTYPE)
    cnt = np.zeros(batch, np.int32)
    check(RT.cudaMemcpy(out.ctypes.data_as(vp), do, sz(out.nbytes), 2), "cudaMemcpy")
    check(RT.cudaMemcpy(cnt.ctypes.data_as(vp), dc, sz(cnt.nbytes), 2), "cudaMemcpy")
    for p in (dm, do, dc):
        check(RT.cudaFree(p), "cudaFree")
    return out.reshape(batch, K), cnt


def agrees(maps, K):
    out, cnt = detect(maps, K)
    for i in range(maps.shape[0]):
        ref = oracle.peaks_ref(np.abs(maps[i]).astype(np.float64), K)
        got = [(int(r["t"]), int(r["s"]), float(r["value"])) for r in out[i, :cnt[i]]]
        if got != ref:
            return False
    return True


rng = np.random.default_rng(11)
K = 16
ok1 = agrees(rng.standard_normal((4, 256, 256)).astype(np.float32), K)
check(RT.cudaDeviceReset(), "cudaDeviceReset")          # new context: new scratch address
ok2 = agrees(rng.standard_normal((4, 256, 256)).astype(np.float32), K)
check(RT.cudaDeviceReset(), "cudaDeviceReset")
print("OK" if ok1 and ok2 else f"MISMATCH {ok1} {ok2}")
