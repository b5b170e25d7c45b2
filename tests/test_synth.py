"""The seeded input generator: deterministic, seed-sensitive, well formed."""
import numpy as np

from paper_1509_04232_gb300 import synth


def test_deterministic_and_seed_sensitive():
    a = synth.voronoi_frame(64, 48, 10, 6.0, 5)
    b = synth.voronoi_frame(64, 48, 10, 6.0, 5)
    c = synth.voronoi_frame(64, 48, 10, 6.0, 6)
    np.testing.assert_array_equal(a, b)
    assert np.mean(a != c) > 0.5


def test_noise_free_regions_are_piecewise_constant():
    img = synth.voronoi_frame(80, 60, 7, 0.0, 11, grad_max=0.0)
    colours = np.unique(img.reshape(-1, 3), axis=0)
    assert 1 <= len(colours) <= 7


def test_rgba_has_opaque_alpha_and_same_rgb():
    rgb = synth.voronoi_frame(33, 17, 5, 8.0, 3)
    rgba = synth.voronoi_frame(33, 17, 5, 8.0, 3, channels=4)
    np.testing.assert_array_equal(rgba[..., :3], rgb)
    assert np.all(rgba[..., 3] == 255)


def test_video_frames_move_and_frame_zero_is_still():
    f0 = synth.video_frame(0, 96, 64)
    f1 = synth.video_frame(1, 96, 64)
    still = synth.voronoi_frame(96, 64, 400, 6.0, synth.seed_of(4, 0))
    np.testing.assert_array_equal(f0, still)
    assert np.mean(f0 != f1) > 0.3


def test_mixed_batch_specs():
    specs = synth.mixed_batch_specs(256)
    assert len(specs) == 256
    sizes = [(w, h) for w, h, _, _ in specs]
    for wh in synth.MIXED_SIZES:
        assert sizes.count(wh) == 64
    assert {s for _, _, s, _ in specs} == {8, 16, 32}
    assert {m for _, _, _, m in specs} == {5.0, 10.0, 20.0}
