"""The seeded input recipes (paper_1509_02468_gb300/synth.py) produce what their docstrings
state: the 1D signal's 12 pieces of at least 16 samples and its noise, the polygon image's
range and noise, the block start, and the sizes of the 256-instance mixed batch
(36.7 M samples).  CPU only."""
import numpy as np
import pytest

from paper_1509_02468_gb300 import synth


def test_signal_1d_pieces_levels_and_noise():
    clean, noisy = synth.signal_1d(4096, 1)
    jumps = np.flatnonzero(np.diff(clean) != 0) + 1
    edges = np.concatenate(([0], jumps, [clean.size]))
    assert len(edges) - 1 == 12                                   # 12 constant pieces
    assert np.diff(edges).min() >= 16                             # at least 16 samples each
    assert clean.min() >= 0.0 and clean.max() <= 1.0              # levels U[0, 1]
    assert np.std(noisy - clean) == pytest.approx(0.1, rel=0.05)  # N(0, 0.1^2)
    again = synth.signal_1d(4096, 1)
    assert np.array_equal(again[1], noisy)                        # seeded
    lin_clean, _ = synth.signal_1d(600, 3, segments=4, kind="linear")
    # ramps: the slope changes only next to the 3 breakpoints (rounding aside)
    assert np.count_nonzero(np.abs(np.diff(lin_clean, 2)) > 1e-12) <= 2 * 3


def test_polygon_image_range_noise_and_layout():
    clean, noisy = synth.polygon_image(300, 200, 2)
    assert clean.shape == (300, 200) and noisy.dtype == np.float32
    assert clean.min() >= 0.0 and clean.max() <= 2.0              # a + b (u.p)/side, levels U[0, 1]
    assert np.std(noisy.astype(np.float64) - clean) == pytest.approx(0.05, rel=0.05)
    # polygons painted over the gradient: many pixels sit exactly on a few constant levels
    vals, counts = np.unique(clean, return_counts=True)
    assert counts.max() > 0.01 * clean.size
    assert np.array_equal(synth.polygon_image(300, 200, 2)[1], noisy)


def test_block_start_columns():
    x0 = np.linspace(0, 1, 5000)
    X = synth.block_start(x0, 8, seed=2, dtype=np.float32)
    assert X.shape == (5000, 8) and X.dtype == np.float32
    np.testing.assert_array_equal(X[:, 0], x0.astype(np.float32))
    rest = X[:, 1:].astype(np.float64)
    assert abs(rest.mean()) < 0.02 and rest.std() == pytest.approx(1.0, rel=0.02)


def test_mixed_batch_sizes():
    sizes = synth.batch_sizes(4)
    assert len(sizes) == 256
    imgs = [s for s in sizes if s[0] == 2]
    sigs = [s for s in sizes if s[0] == 1]
    assert len(imgs) == 192 and len(sigs) == 64
    assert all(64 <= h <= 1024 and 64 <= w <= 1024 for _, h, w in imgs)
    assert all(ny == 1 and 1000 <= n <= 1_000_000 for _, ny, n in sigs)
    total = sum(h * w for _, h, w in sizes)
    assert total == pytest.approx(36.7e6, rel=0.01)               # the batch's 36.7 M samples
