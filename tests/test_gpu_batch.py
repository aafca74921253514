"""Mixed-size batches (ft_batch_*): packed layout, one graph launch, autotuner.

Without tuning every group uses the same kernels as a single-shape plan, so the
batch must reproduce per-image ft_forward / ft_peaks bit for bit; tuned variants
are checked against the FP64 oracle instead."""
import json

import numpy as np
import pytest

import oracle
from paper_1904_09409_gb300 import synth
from tests import _gpu

pytestmark = pytest.mark.gpu
SHAPES = [(64, 64), (96, 128), (64, 64), (128, 96), (192, 256), (96, 128), (256, 192), (64, 64),
          (48, 72)]   # 48 x 72: no fixed-length schedule, generic kernels
TOP_K = 5


@pytest.fixture(scope="module")
def torch():
    return _gpu.torch_cuda()


def images(seed=0):
    return [synth.varlen_image(seed * 100 + i, h, w).img for i, (h, w) in enumerate(SHAPES)]


def individual(imgs):
    from paper_1904_09409_gb300 import funnel as f
    maps, peaks = [], []
    for img in imgs:
        h, w = img.shape
        with f.Plan(h, w, w, h) as plan:
            m = _gpu.forward(plan, img[None])
            maps.append(m[0])
            peaks.append(_gpu.peaks(plan, m, TOP_K)[1][0])
    return maps, peaks


def run_batch(torch, b, imgs, **kw):
    from paper_1904_09409_gb300 import funnel as f
    x = torch.from_numpy(b.pack(imgs)).cuda()
    m = torch.full((b.map_total,), float("nan"), device="cuda")
    out = torch.zeros(b.n * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(b.n, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(x, m, TOP_K, out=out, count=cnt, stream=s, **kw)
    s.synchronize()
    maps = b.unpack_maps(m.cpu().numpy())
    recs = out.cpu().numpy().view(f.PEAK_DTYPE).reshape(b.n, TOP_K)
    cnts = cnt.cpu().numpy()
    peaks = [None] * b.n
    for j, i in enumerate(b.order):
        peaks[i] = recs[j, :cnts[j]]
    return maps, peaks, (x, m, out, cnt, s)


def test_batch_matches_individual_plans(torch):
    from paper_1904_09409_gb300 import funnel as f
    imgs = images()
    ref_maps, ref_peaks = individual(imgs)
    with f.Batch(SHAPES) as b:
        assert sorted(b.order.tolist()) == list(range(len(SHAPES)))
        assert sum(g["count"] for g in b.groups()) == len(SHAPES)
        maps, peaks, _ = run_batch(torch, b, imgs)
    for i in range(len(SHAPES)):
        assert np.array_equal(maps[i], ref_maps[i]), i
        assert np.array_equal(peaks[i], ref_peaks[i]), i


def test_graph_replay(torch):
    from paper_1904_09409_gb300 import funnel as f
    imgs1, imgs2 = images(1), images(2)
    ref_maps, ref_peaks = individual(imgs2)
    with f.Batch(SHAPES) as b:
        maps1, _, bufs = run_batch(torch, b, imgs1, graph=True)
        x, m, out, cnt, s = bufs
        # replay with new contents in the same buffers
        x.copy_(torch.from_numpy(b.pack(imgs2)).cuda())
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            b.run(x, m, TOP_K, out=out, count=cnt, stream=s, graph=True)
        s.synchronize()
        maps2 = b.unpack_maps(m.cpu().numpy())
        recs = out.cpu().numpy().view(f.PEAK_DTYPE).reshape(b.n, TOP_K)
        cnts = cnt.cpu().numpy()
        for j, i in enumerate(b.order):
            assert np.array_equal(maps2[i], ref_maps[i])
            assert np.array_equal(recs[j, :cnts[j]], ref_peaks[i])
    for i in range(len(SHAPES)):
        h, w = SHAPES[i]
        assert _gpu.rel_l2(maps1[i], oracle.funnel_ref(imgs1[i], w, h)) <= 1e-5


def test_autotuner_and_cache(torch, tmp_path):
    from paper_1904_09409_gb300 import funnel as f
    cache = str(tmp_path / "tune.json")
    imgs = images(3)
    with f.Batch(SHAPES, tune_cache=cache) as b:
        maps, _, _ = run_batch(torch, b, imgs, tune=True)
        tuned = {(g["H"], g["W"]): g["variant"] for g in b.groups()}
        assert all(0 <= v <= 4 for v in tuned.values())
        assert all(g["tuned_ms"] > 0 for g in b.groups())
    for i in range(len(SHAPES)):
        h, w = SHAPES[i]
        assert _gpu.rel_l2(maps[i], oracle.funnel_ref(imgs[i], w, h)) <= 1e-5
    entries = json.load(open(cache))
    assert len(entries) == len(tuned)
    with f.Batch(SHAPES, tune_cache=cache) as b2:          # choices come back from the cache
        assert {(g["H"], g["W"]): g["variant"] for g in b2.groups()} == tuned


LARGE_SHAPES = [(2048, 2048), (1536, 1536), (2048, 1536), (1536, 2048), (128, 2048), (2048, 128),
                (768, 1536), (1536, 768), (2048, 2048)]


def test_batch_with_1536_and_2048_matches_oracle(torch):
    """The mixed-size workload's longest sides (the fixed-length schedules of
    1536 = 4^4 * 2 * 3 and 2048 = 16 * 16 * 8) in one batch: every map against
    the FP64 oracle, every peak list against the oracle's list procedure on the
    same FP32 map."""
    from paper_1904_09409_gb300 import funnel as f
    imgs = [synth.varlen_image(500 + i, h, w).img for i, (h, w) in enumerate(LARGE_SHAPES)]
    with f.Batch(LARGE_SHAPES) as b:
        x = torch.from_numpy(b.pack(imgs)).cuda()
        m = torch.full((b.map_total,), float("nan"), device="cuda")
        out = torch.zeros(b.n * TOP_K * f.PEAK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(b.n, dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            b.run(x, m, TOP_K, out=out, count=cnt, stream=s)
        s.synchronize()
        maps = b.unpack_maps(m.cpu().numpy())
        recs = out.cpu().numpy().view(f.PEAK_DTYPE).reshape(b.n, TOP_K)
        cnts = cnt.cpu().numpy()
        order = list(b.order)
    for j, i in enumerate(order):
        h, w = LARGE_SHAPES[i]
        assert _gpu.rel_l2(maps[i], oracle.funnel_ref(imgs[i], w, h)) <= 1e-5, (h, w)
        got = [(int(r["t"]), int(r["s"]), float(r["value"])) for r in recs[j, :cnts[j]]]
        assert got == oracle.peaks_ref(np.abs(maps[i]).astype(np.float64), TOP_K), (h, w)
