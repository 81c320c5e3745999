"""The synthetic inputs (host only): shapes, ranges, masks and query sets as
the input recipe states them, and determinism (the same seed gives the same
arrays, so every test and bench line sees the same inputs)."""
import numpy as np

import oracle as O
from paper_1712_06326_gb300 import synth


def test_sines2d_recipe():
    g, m = synth.sines2d(128)
    assert g.shape == (128, 128, 1) and g.dtype == np.float32 and m.shape == (128, 128)
    assert g.min() >= 0.0 and g.max() <= 1.0
    # centred 24^2 hole, rows and columns 52..75
    assert (m == 0).sum() == 576 and np.all(m[52:76, 52:76] == 0)
    assert len(O.dict_extract(m, 9)) == 13376
    g2, m2 = synth.sines2d(128)
    assert np.array_equal(g, g2) and np.array_equal(m, m2)


def test_voronoi2d_bench_workload():
    g, m = synth.voronoi2d(1024, cfg=2)
    assert g.shape == (1024, 1024, 3) and g.dtype == np.float32
    assert g.min() >= 0.0 and g.max() <= 1.0
    unknown = (m == 0).mean()
    assert 0.10 <= unknown < 0.13  # discs are added until at least 10 % are unknown
    assert len(O.dict_extract(m, 11)) == 901592
    t = synth.front_targets(m, 11, cap=65536, cfg=2)
    assert t.shape == (3597, 2) and t.dtype == np.int32
    assert t.min() >= 5 and t[:, 0].max() <= 1018 and t[:, 1].max() <= 1018
    lin = t[:, 1].astype(np.int64) * 1024 + t[:, 0]
    assert np.all(np.diff(lin) > 0)  # raster order, no duplicates
    g2, m2 = synth.voronoi2d(1024, cfg=2)
    assert np.array_equal(g, g2) and np.array_equal(m, m2)


def test_front_targets_touch_the_hole():
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)
    K, r = 7, 3
    for x, y in synth.front_targets(m, K):
        box = m[y - r:y + r + 1, x - r:x + r + 1]
        assert box.shape == (K, K) and 0 < box.sum() < K * K  # partly known, partly not


def test_spheres3d_blocks_and_range():
    g, m = synth.spheres3d(64, block=8, missing=0.15)
    assert g.shape == (64, 64, 64, 1) and m.shape == (64, 64, 64)
    assert g.min() >= 0.0 and g.max() <= 1.0
    # the mask is a union of aligned 8^3 blocks, 15 % of them
    blocks = m.reshape(8, 8, 8, 8, 8, 8).transpose(0, 2, 4, 1, 3, 5).reshape(512, 512)
    assert np.all((blocks.min(1) == blocks.max(1)))
    assert (blocks[:, 0] == 0).sum() == round(0.15 * 512)


def test_batch_sizes_log_uniform_range():
    sizes = synth.batch_sizes(256, cfg=4)
    assert len(sizes) == 256
    w = np.array([a for a, _ in sizes])
    h = np.array([b for _, b in sizes])
    assert w.min() >= 256 and w.max() <= 2048 and h.min() >= 256 and h.max() <= 2048
    # log-uniform: about half of each side below the geometric middle 724
    assert 0.35 < (w < 724).mean() < 0.65 and 0.35 < (h < 724).mean() < 0.65
    assert synth.batch_sizes(256, cfg=4) == sizes
    g, m, t = synth.batch_case(3, (300, 260), 9, 64)
    assert g.shape == (260, 300, 3) and m.shape == (260, 300) and 0 < len(t) <= 64
