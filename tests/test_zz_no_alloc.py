"""ft_peaks_noalloc, the peak detection for callers that cannot allocate device
memory (stream capture, fixed memory budgets, foreign allocators), checked
against ft_peaks through the C ABI.  Peak lists are integer index work, so the
two entry points must agree exactly.  This file is collected last on purpose:
it must pass both alone in a fresh process and after every other test."""
import ctypes

import numpy as np
import pytest

from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return _gpu.torch_cuda()


def _call_noalloc(L, m, Hp, S, batch, K, thr, out, cnt):
    return L.ft_peaks_noalloc(ctypes.c_void_p(m.data_ptr()), Hp, S, batch, K, ctypes.c_float(thr),
                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(cnt.data_ptr()),
                              ctypes.c_void_p(torch_stream()))


def torch_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("Hp,S,batch,K,thr", [(1024, 1024, 8, 32, float("-inf")),
                                              (96, 216, 3, 64, 1.5),
                                              (256, 192, 2, 600, float("-inf"))])
def test_noalloc_matches_ft_peaks_twice(torch, Hp, S, batch, K, thr):
    from paper_1904_09409_gb300 import funnel as f
    L = f.lib()
    rng = np.random.default_rng(Hp + S + K)
    with f.Plan(Hp, S, S, Hp) as plan:
        for call in range(2):                       # two calls in a row, different maps
            maps = rng.standard_normal((batch, Hp, S)).astype(np.float32)
            if call == 1:
                maps = np.round(maps * 2.0)             # ties on the second call
            m = torch.from_numpy(maps).cuda()
            ref_out, ref_cnt = f.ft_peaks(plan, m, K, thr)
            out = torch.full((batch * K * f.PEAK_DTYPE.itemsize,), 0xAB, dtype=torch.uint8, device="cuda")
            cnt = torch.full((batch,), -1, dtype=torch.int32, device="cuda")
            assert _call_noalloc(L, m, Hp, S, batch, K, thr, out, cnt) == f.FT_OK
            torch.cuda.synchronize()
            assert torch.equal(cnt, ref_cnt)
            assert torch.equal(out, ref_out)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    from paper_1904_09409_gb300 import funnel as f
    L = f.lib()
    m = torch.zeros((1, 8, 8), device="cuda")
    out = torch.empty(1024 * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    # 4096 x 8192 maps, 64 of them, top-512: far beyond FT_NOALLOC_SCRATCH_BYTES; the
    # size check runs before any pointer is used
    st = _call_noalloc(L, m, 4096, 8192, 64, 512, 0.0, out, cnt)
    assert st == f.FT_ERR_UNSUPPORTED_SIZE
    assert b"FT_NOALLOC_SCRATCH_BYTES" in L.ft_last_error()
    with pytest.raises(f.FunnelError, match="FT_NOALLOC_SCRATCH_BYTES"):
        # 2 maps of 2048 x 8192 with top-512: 2 x 64 x 128 tiles x 512 keys x 8 B = 64 MiB
        f.ft_peaks_noalloc(torch.zeros((2, 2048, 8192), device="cuda"), 512)


def test_noalloc_after_device_reset():
    """The scratch array's device address belongs to one CUDA context; after
    cudaDeviceReset the next call must look it up again in the new context.
    Runs in a child process (the reset would invalidate this process's torch
    memory)."""
    import os
    import subprocess
    import sys
    _gpu.torch_cuda()                                   # builds the library if needed
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_noalloc_reset_child.py")
    r = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK"), r.stdout + r.stderr


def test_noalloc_inside_stream_capture(torch):
    """One warm-up call, then a call captured into a CUDA graph on a static map;
    the graph replayed on new map contents gives ft_peaks' result byte for byte."""
    from paper_1904_09409_gb300 import funnel as f
    Hp, S, batch, K = 512, 384, 3, 40
    rng = np.random.default_rng(3)
    m = torch.from_numpy(rng.standard_normal((batch, Hp, S)).astype(np.float32)).cuda()
    out = torch.zeros(batch * K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(batch, dtype=torch.int32, device="cuda")
    f.ft_peaks_noalloc(m, K, out=out, count=cnt)        # warm-up before any capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        f.ft_peaks_noalloc(m, K, out=out, count=cnt)
    new = rng.standard_normal((batch, Hp, S)).astype(np.float32)
    m.copy_(torch.from_numpy(new).cuda())
    out.fill_(0xAB)
    cnt.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    with f.Plan(Hp, S, S, Hp) as plan:
        ref_out, ref_cnt = f.ft_peaks(plan, m, K)
        torch.cuda.synchronize()
    assert torch.equal(cnt, ref_cnt)
    assert torch.equal(out, ref_out)
