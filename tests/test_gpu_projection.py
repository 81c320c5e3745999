"""The FP32 projections of 2-D indices (Sec. II.A: y = B^T (x - mu) of every
dictionary patch's subset, per index) on the GPU (needs a GB300): from a common
imported basis, the projections, quantisers, keys and sorted arrays must equal
the oracle's bit for bit -- over non-square images, grey, RGB and 8-channel
grids, odd and even numbers of axes (5, 8, 12, 16), patches of 7 to 15 pixels
a side, and masks whose holes cover nearly half of the image."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_06326_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1712_06326_gb300 import sfc

    torch.cuda.set_device(0)
    sfc.sfc_status()
    return sfc


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def random_basis(K, ch, C_, D, seed):
    s = O.subsets(2, K, 0.6, C_).shape[1] * ch
    rng = np.random.default_rng(seed)
    B = rng.normal(0.0, 0.2, (C_, s, D)).astype(np.float32)
    mu = rng.uniform(0.0, 1.0, (C_, s)).astype(np.float32)
    return B, mu


def check_projection(S, g, m, K, C_, D, bits, seed):
    ch = g.shape[2]
    B, mu = random_basis(K, ch, C_, D, seed)
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=8, basis=B, mean=mu,
                           keep_intermediates=1)
    ex = S.sfc_index_export(ix, proj=True)
    ix.close()
    assert S.sfc_status() == 0
    oix = O.build_index(g, m, K, C_, D, bits, basis=B, mean=mu)
    assert np.array_equal(oix["dict"], ex["dict"])
    assert np.array_equal(oix["proj"].view(np.uint32), ex["proj"].view(np.uint32))
    assert np.array_equal(oix["lo"], ex["lo"]) and np.array_equal(oix["scale"], ex["scale"])
    assert np.array_equal(oix["keys"], ex["keys"])
    assert np.array_equal(oix["skeys"], ex["skeys"]) and np.array_equal(oix["sids"], ex["sids"])
    return ex


def test_rgb_non_square_odd_axes(S):
    # 150 x 97 pixels, D = 5 (an odd number of axes: one unpaired chain)
    g, m = synth.voronoi2d(150, 97, cfg=2, seed_sub=71)
    check_projection(S, g, m, K=9, C_=3, D=5, bits=12, seed=1)


def test_grey_sixteen_axes(S):
    # 16 axes of 7 x 7 grey patches (s = 29)
    g, m = synth.sines2d(131)
    g = np.ascontiguousarray(g[:77])
    m = np.ascontiguousarray(m[:77])
    check_projection(S, g, m, K=7, C_=2, D=16, bits=4, seed=2)


def test_rgb_large_patch_twelve_axes(S):
    # 12 axes of 15 x 15 RGB patches (s = 405)
    g, m = synth.voronoi2d(120, 90, cfg=2, seed_sub=72)
    check_projection(S, g, m, K=15, C_=2, D=12, bits=5, seed=3)


def test_large_holes(S):
    # holes over 45 % of the pixels: whole blocks of entries are missing
    g, m = synth.voronoi2d(200, cfg=2, seed_sub=73, coverage=0.45)
    ex = check_projection(S, g, m, K=7, C_=4, D=8, bits=16, seed=4)
    assert len(ex["dict"]) < 0.55 * 194 * 194


def test_eight_channels(S):
    # 15 x 15 patches of 8 channels (s = 1,080: the basis tables take 26 KB
    # of shared memory per block)
    g0, m = synth.voronoi2d(70, 66, cfg=2, seed_sub=74, coverage=0.05)
    g = np.ascontiguousarray(np.concatenate([g0, g0[..., ::-1], g0[..., :2] * 0.5], axis=2))
    assert g.shape[2] == 8
    check_projection(S, g, m, K=15, C_=1, D=4, bits=10, seed=5)
