"""Mixed-size batches (ft_batch_*): packed layout, grouped kernels (one launch
per stage over every shape with a fixed-length schedule up to 2048), per-shape
plans for the other shapes, one graph launch, autotuner.

The grouped kernels run the same FFT arithmetic per transform as a single-shape
plan (only the transforms per block differ), so the batch must reproduce
per-image ft_forward / ft_peaks bit for bit, in every configuration of the
autotuner; tuned plan variants are checked against the FP64 oracle instead."""
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
        plan_groups = [g for g in b.groups() if g["variant"] >= 0]
        assert all(0 <= g["variant"] <= 4 and g["tuned_ms"] > 0 for g in plan_groups)
        # the grouped kernels: 8 configurations timed, the fastest kept
        ms = b.tune_ms()
        assert len(ms) == 8 and all(v > 0 for v in ms.values())
        cfg = b.config()
        chosen = (cfg["r2c_threads"], cfg["rows_threads"], cfg["c2r_threads"])
        assert ms[chosen] == min(ms.values())
    for i in range(len(SHAPES)):
        h, w = SHAPES[i]
        assert _gpu.rel_l2(maps[i], oracle.funnel_ref(imgs[i], w, h)) <= 1e-5
    entries = json.load(open(cache))
    assert len(entries) == len(plan_groups) + 1             # one entry for the grouped kernels
    with f.Batch(SHAPES, tune_cache=cache) as b2:          # choices come back from the cache
        assert {(g["H"], g["W"]): g["variant"] for g in b2.groups()} == tuned
        c2 = b2.config()
        assert (c2["r2c_threads"], c2["rows_threads"], c2["c2r_threads"]) == chosen


SIZES = (128, 192, 256, 384, 512, 768, 1024, 1536, 2048)


def test_grouped_kernels_every_configuration_bit_exact(torch):
    """Shapes drawn from the mixed-size workload's sizes (both sides from
    {128 ... 2048}, so every image runs in the grouped kernels: 4 launches)
    plus two shapes on plans of their own: in each of the 8 configurations the
    maps and peak lists equal those of per-image plans bit for bit."""
    from paper_1904_09409_gb300 import funnel as f
    rng = np.random.default_rng(77)
    shapes = [(int(rng.choice(SIZES[:7])), int(rng.choice(SIZES[:7]))) for _ in range(18)]
    shapes += [(2048, 256), (192, 1536), (128, 128), (64, 64), (48, 72)]
    imgs = [synth.varlen_image(700 + i, h, w).img for i, (h, w) in enumerate(shapes)]
    ref_maps, ref_peaks = individual(imgs)
    with f.Batch(shapes) as b:
        cfg = b.config()
        assert cfg["grouped_images"] == len(shapes) - 2 and cfg["plan_groups"] == 2
        for c in range(8):
            r2c, rows, c2r = (256, 512)[c >> 2 & 1], (128, 256)[c >> 1 & 1], (256, 512)[c & 1]
            b.set_config(r2c, rows, c2r)
            maps, peaks, _ = run_batch(torch, b, imgs)
            for i in range(len(shapes)):
                assert np.array_equal(maps[i], ref_maps[i]), (c, shapes[i])
                assert np.array_equal(peaks[i], ref_peaks[i]), (c, shapes[i])
        with pytest.raises(f.FunnelError):
            b.set_config(384, 128, 256)
    with f.Batch([s for s in shapes if s[0] >= 128 and s[1] >= 128]) as b:
        assert b.config()["plan_groups"] == 0
        assert b.launches(TOP_K) == 4 and b.launches(0) == 3


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
