"""ft_detect_batches: consecutive batches as one pipeline (step 1 of batch j + 1
beside the peak pass of batch j).  The records and counts must equal those of
one ft_detect call per batch bit for bit, with the pipeline on and off, at the
benchmark's image size and at sizes that take the non-pipelined path; the
records are also checked against the FP64 oracle's peak detection of the
FP32 map.  A race between the peak pass of batch j and step 4 of batch j + 1
(both touch the shared map buffer) would change the records of batch j, so
every case gives each batch different images."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1904_09409_gb300 import synth
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return _gpu.torch_cuda()


def _batches(nb, batch, side, seed):
    return [synth.batch_1024(batch, start=seed + j * batch, side=side) for j in range(nb)]


def _per_call(plan, xs, K, thr):
    from paper_1904_09409_gb300 import funnel as f
    import torch as T
    b = xs[0].shape[0]
    m = T.empty((b, plan.Hp, plan.S), device="cuda")
    outs, cnts = [], []
    for x in xs:
        out, cnt = f.ft_detect(plan, x, m, K, thr)
        outs.append(out.clone())
        cnts.append(cnt.clone())
    T.cuda.synchronize()
    return T.cat(outs), T.cat(cnts), m.clone()


@pytest.mark.parametrize("side,nb,batch,K,thr", [(1024, 6, 16, 32, float("-inf")), (1024, 3, 5, 7, 0.0),
                                                 (1024, 1, 4, 32, float("-inf")), (256, 5, 9, 32, 1.0),
                                                 (512, 4, 3, 100, float("-inf"))])
@pytest.mark.parametrize("pdl", ["1", "0"])
def test_detect_batches_equals_detect_calls(torch, monkeypatch, side, nb, batch, K, thr, pdl):
    from paper_1904_09409_gb300 import funnel as f
    monkeypatch.setenv("FT_PDL", pdl)
    xs = [torch.from_numpy(b).cuda() for b in _batches(nb, batch, side, seed=7 * side + nb)]
    with f.Plan(side, side, side, side) as plan:
        ref_out, ref_cnt, ref_map = _per_call(plan, xs, K, thr)
        m = torch.full((batch, side, side), float("nan"), device="cuda")
        out, cnt = f.ft_detect_batches(plan, xs, m, K, thr)
        torch.cuda.synchronize()
        assert torch.equal(cnt, ref_cnt)
        assert torch.equal(out, ref_out)
        assert torch.equal(m, ref_map)                 # the last batch's maps
        if side == 1024 and pdl == "1":
            # the records of the middle batch against the oracle's detection on its FP32 map
            j = nb // 2
            mj = torch.empty_like(m)
            f.ft_forward(plan, xs[j], mj)
            torch.cuda.synchronize()
            recs = f.peaks_to_numpy(out[j * batch * K * f.PEAK_DTYPE.itemsize:], cnt[j * batch:], K)
            for i in (0, batch - 1):
                got = [(int(p["t"]), int(p["s"]), float(p["value"])) for p in recs[i]]
                assert got == oracle.peaks_ref(np.abs(mj[i].cpu().numpy()).astype(np.float64), K, thr), (j, i)


def test_detect_batches_generic_sizes(torch):
    """A size without the pipelined path (no fixed-length schedule): nb ft_detect calls."""
    from paper_1904_09409_gb300 import funnel as f
    rng = np.random.default_rng(3)
    xs = [torch.from_numpy(rng.standard_normal((2, 100, 96)).astype(np.float32)).cuda() for _ in range(3)]
    with f.Plan(100, 96, 96, 192) as plan:
        ref_out, ref_cnt, ref_map = _per_call(plan, xs, 5, float("-inf"))
        m = torch.empty((2, 192, 96), device="cuda")
        out, cnt = f.ft_detect_batches(plan, xs, m, 5)
        torch.cuda.synchronize()
        assert torch.equal(out, ref_out) and torch.equal(cnt, ref_cnt) and torch.equal(m, ref_map)


def test_detect_batches_arguments(torch):
    from paper_1904_09409_gb300 import funnel as f
    L = f.lib()
    x = torch.zeros((2, 64, 64), device="cuda")
    m = torch.empty((2, 64, 64), device="cuda")
    out = torch.empty(2 * 2 * 4 * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.empty(4, dtype=torch.int32, device="cuda")
    with f.Plan(64, 64, 64, 64) as plan:
        def call(ptrs, nb, batch=2, K=4, thr=float("-inf")):
            arr = (ctypes.c_void_p * max(len(ptrs), 1))(*ptrs)
            return L.ft_detect_batches(plan.handle, arr, nb, batch, m.data_ptr(), K, thr, out.data_ptr(),
                                       cnt.data_ptr(), None)
        good = x.data_ptr()
        assert call([good, good], 2) == f.FT_OK
        assert call([good, None], 2) == f.FT_ERR_INVALID_ARG
        assert call([good, good + 4], 2) == f.FT_ERR_INVALID_ARG      # misaligned
        assert call([good], -1) == f.FT_ERR_INVALID_ARG
        assert call([good], 1, K=0) == f.FT_ERR_INVALID_ARG
        assert call([good], 1, thr=float("nan")) == f.FT_ERR_INVALID_ARG
        assert call([], 0) == f.FT_OK
        assert call([good], 1, batch=0) == f.FT_OK
        torch.cuda.synchronize()


@pytest.mark.parametrize("case", ["inverse", "dense"])
def test_detect_batches_fallbacks(torch, monkeypatch, case):
    """The inverse space and the per-tile key pass (FT_PEAKS=dense) take nb
    ft_detect calls instead of the pipeline: the same records, counts and maps."""
    from paper_1904_09409_gb300 import funnel as f
    if case == "dense":
        monkeypatch.setenv("FT_PEAKS", "dense")
        plan = f.Plan(256, 256, 256, 256)
    else:
        plan = f.Plan(256, 192, space="inverse")
    with plan:
        xs = [torch.from_numpy(b[:, :plan.H, :plan.W].copy()).cuda()
              for b in _batches(3, 4, 256, seed=11 if case == "dense" else 13)]
        ref_out, ref_cnt, ref_map = _per_call(plan, xs, 8, float("-inf"))
        m = torch.empty((4, plan.Hp, plan.S), device="cuda")
        out, cnt = f.ft_detect_batches(plan, xs, m, 8)
        torch.cuda.synchronize()
        assert torch.equal(out, ref_out) and torch.equal(cnt, ref_cnt) and torch.equal(m, ref_map)
