"""The seeded input recipe (no GPU): determinism, ranges, and the warp that defines the ground truth."""
import numpy as np

from paper_1402_2020_gb300 import synth


def test_pairs_are_seeded_int8_offsets_inside_the_window():
    for n, S in ((32, 9), (256, 31), (4096, 26)):
        a = synth.pair_table(n, S, seed=5)
        b = synth.pair_table(n, S, seed=5)
        assert a.dtype == np.int8 and a.shape == (n, 4)
        assert np.array_equal(a, b)
        assert np.abs(a.astype(np.int32)).max() <= S // 2
    assert not np.array_equal(synth.pair_table(256, 31, seed=5), synth.pair_table(256, 31, seed=6))


def test_pair_spread_follows_sigma():
    # the rounded Gaussian truncated at |offset| <= S // 2: sigma S / 5 = 6.2 at S = 31 gives a spread just
    # under 6.2; an explicit sigma (the paper's 4 at S = 26) is honoured the same way
    p = synth.pair_table(4096, 31, seed=1).astype(np.float64)
    assert 5.6 < p.std() < 6.3 and abs(p.mean()) < 0.2
    q = synth.pair_table(4096, 26, sigma=4.0, seed=1).astype(np.float64)
    assert 3.8 < q.std() < 4.2


def test_stereo_pair_is_deterministic_and_in_range():
    l1, r1, g1 = synth.stereo_pair(120, 50, 24, seed=9)
    l2, r2, g2 = synth.stereo_pair(120, 50, 24, seed=9)
    assert l1.dtype == np.uint8 and l1.shape == (50, 120, 3) and r1.shape == l1.shape
    assert g1.dtype == np.int32 and g1.shape == (50, 120)
    assert np.array_equal(l1, l2) and np.array_equal(r1, r2) and np.array_equal(g1, g2)
    assert g1.min() >= 0 and g1.max() <= 23
    l3, _, _ = synth.stereo_pair(120, 50, 24, seed=10)
    assert not np.array_equal(l1, l3)


def test_right_view_is_the_forward_warp_with_the_larger_disparity_winning():
    w, h, dmax = 64, 12, 16
    left, right, gt = synth.stereo_pair(w, h, dmax, seed=3)
    hits = 0
    for y in range(h):
        best = {}
        for x in range(w):
            xr = x - int(gt[y, x])
            if xr >= 0 and (xr not in best or (gt[y, x], x) > best[xr]):
                best[xr] = (int(gt[y, x]), x)
        for xr, (_, x) in best.items():
            assert np.array_equal(right[y, xr], left[y, x]), (y, xr, x)
            hits += 1
    assert hits > 0.5 * w * h


def test_radiometric_change_is_monotone_and_identity_at_unit_settings():
    v = np.arange(256, dtype=np.uint8).reshape(1, 256, 1).repeat(3, axis=2)
    assert np.array_equal(synth.radiometric_fixed(v, 1.0, 1.0), v)
    for g, gamma in ((0.5, 0.7), (2.0, 1.4), (1.0, 1.4)):
        out = synth.radiometric_fixed(v, g, gamma)[0, :, 0].astype(np.int32)
        assert (np.diff(out) >= 0).all() and out[0] == 0
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, size=(8, 8, 3)).astype(np.uint8)
    out = synth.radiometric_fixed(img, 1.0, 1.0, off=(10.0, -10.0, 0.0)).astype(np.int32)
    assert np.array_equal(out[..., 0], np.minimum(img[..., 0].astype(np.int32) + 10, 255))
    assert np.array_equal(out[..., 1], np.maximum(img[..., 1].astype(np.int32) - 10, 0))


def test_shifted_pair_has_a_constant_shift():
    left, right = synth.shifted_pair(50, 7, 6, seed=2)
    assert np.array_equal(right[:, : 50 - 6], left[:, 6:])


def test_batch_shapes_follow_the_stated_ranges():
    shapes = synth.batch_shapes(64, seed=3)
    assert len(shapes) == 64 and shapes == synth.batch_shapes(64, seed=3)
    for w, h, d, s in shapes:
        assert 320 <= w <= 1920 and 240 <= h <= 1080 and d in (64, 128, 192, 256)
    assert len({s for _, _, _, s in shapes}) == 64
