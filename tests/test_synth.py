"""The seeded generator: determinism, shapes and content ranges."""
import numpy as np

from paper_1904_09409_gb300 import synth


def test_single_256_is_deterministic():
    a, b = synth.single_256(), synth.single_256()
    assert a.img.dtype == np.float32 and a.img.shape == (256, 256)
    assert np.array_equal(a.img, b.img)
    assert len(a.lines) == 3 and all(l.kind == "ridge" and l.sigma == 1.5 for l in a.lines)
    assert all(-1 <= l.k <= 1 and 0 <= l.b_c < 256 for l in a.lines)


def test_mixed_content_ranges():
    for i in range(6):
        s = synth.mixed_image(synth.WL_BATCH_1024, i, 128, 160)
        assert s.img.shape == (128, 160)
        assert 1 <= len(s.lines) <= 20
        assert 0.05 <= s.noise_sigma <= 0.5
        for l in s.lines:
            if l.kind == "ridge":
                assert 1.0 <= l.sigma <= 3.0 and l.amp == 1.0
            else:
                assert 0.3 <= l.amp <= 1.0


def test_distinct_seeds_give_distinct_images():
    a = synth.mixed_image(synth.WL_BATCH_1024, 0, 64, 64).img
    b = synth.mixed_image(synth.WL_BATCH_1024, 1, 64, 64).img
    c = synth.mixed_image(synth.WL_GRAD_512, 0, 64, 64).img
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_varlen_shapes_from_the_size_set():
    shapes = synth.varlen_shapes(64)
    assert len(shapes) == 64
    assert all(h in synth.VARLEN_SIDES and w in synth.VARLEN_SIDES for h, w in shapes)


def test_ridge_profile_peak_on_the_line():
    img = np.zeros((64, 64))
    synth.render_ridge(img, 0.0, 20.0, 1.5, 1.0)
    assert np.allclose(img[20], 1.0) and np.allclose(img[21], np.exp(-1 / (2 * 1.5 ** 2)))


def test_step_edges_match_the_half_plane_definition():
    """compose() paints step edges through first-row increments; the result is
    the half-plane sum of render_step."""
    rng = synth.rng_for(99, 0)
    lines = synth.draw_lines(rng, 12, 64, 0.0, (1.0, 1.0), 1.0, (0.3, 1.0))
    got = synth.compose(synth.rng_for(99, 1), 64, 80, lines, 0.0, 0.0, 0.25).img
    ref = np.full((64, 80), 0.25)
    for ln in lines:
        synth.render_step(ref, ln.k, ln.b_c, ln.amp)
    assert np.max(np.abs(got - ref)) <= 1e-6
