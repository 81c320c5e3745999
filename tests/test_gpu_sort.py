"""The index sort (Sec. II.C: the dictionary in z-order) on the GPU (needs a
GB300): the sample sort taken by dictionaries of up to 2^20 entries, its
fallback to the LSD radix sort (an index with a bucket above the capacity),
and the LSD sort itself all give the oracle's stable sort of the index's keys
bit for bit -- on RGB and grey images, a 3-D volume, dictionaries of one
bucket, of two, with ragged tiles, and a constant image whose keys are all
equal (the order is then the ids' alone)."""
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
    yield sfc
    sfc.sfc_debug_sort(False, 0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def sorted_arrays(S, g, m, mode, **params):
    """(keys, skeys, sids) of a build with the given sort: 'sample', 'lsd' or
    'fallback' (sample sort with bucket capacity 64)."""
    S.sfc_debug_sort(mode == "lsd", 64 if mode == "fallback" else 0)
    try:
        ix = S.sfc_index_build(dev(g), dev(m), keep_intermediates=1, **params)
        ex = S.sfc_index_export(ix, proj=True)
        ix.close()
    finally:
        S.sfc_debug_sort(False, 0)
    assert S.sfc_status() == 0
    return ex


def check_all_modes(S, g, m, **params):
    ref = None
    for mode in ("sample", "lsd", "fallback"):
        ex = sorted_arrays(S, g, m, mode, **params)
        if ref is None:
            ref = ex
            for c in range(ex["keys"].shape[0]):
                sk, si = O.sort(ex["keys"][c])
                assert np.array_equal(sk, ex["skeys"][c]) and np.array_equal(si, ex["sids"][c]), c
        else:
            assert np.array_equal(ex["keys"], ref["keys"])
            assert np.array_equal(ex["skeys"], ref["skeys"]), mode
            assert np.array_equal(ex["sids"], ref["sids"]), mode
    return ref


def test_sort_rgb_many_buckets(S):
    g, m = synth.voronoi2d(256, cfg=2, seed_sub=31)
    ex = check_all_modes(S, g, m, K=9, curves=4, dims=8, bits=16, window=32, pca_sample=0)
    assert len(ex["dict"]) > 32 * 1024  # at least 32 buckets, several count tiles


def test_sort_grey_shifts_ragged(S):
    g, m = synth.sines2d(96)
    C_, D, bits = 3, 5, 9
    shifts = np.random.default_rng(5).integers(0, 1 << bits, (C_, D)).astype(np.int32)
    ex = check_all_modes(S, g, m, K=7, curves=C_, dims=D, bits=bits, window=16, pca_sample=0, shifts=shifts)
    assert len(ex["dict"]) % 4096 != 0


def test_sort_one_and_two_buckets(S):
    # N <= 512: a single bucket (no splitters); 512 < N <= 1024: two
    for side in (26, 32):
        g = np.random.default_rng(side).random((side, side, 3)).astype(np.float32)
        m = np.ones((side, side), np.uint8)
        m[side // 2 - 2:side // 2 + 2, side // 2 - 2:side // 2 + 2] = 0
        ex = check_all_modes(S, g, m, K=5, curves=2, dims=4, bits=8, window=8, pca_sample=0)
        n = len(ex["dict"])
        assert (n <= 512) if side == 26 else (512 < n <= 1024)


def test_sort_3d(S):
    g, m = synth.spheres3d(28, block=4, missing=0.1, seed_sub=7)
    check_all_modes(S, g, m, K=5, curves=4, dims=6, bits=12, window=16, pca_sample=0)


def test_sort_all_keys_equal(S):
    # a constant image: every patch projects to the same point; the basis is
    # imported (a constant image has no principal directions of its own)
    g0, m0 = synth.voronoi2d(64, cfg=2, seed_sub=32)
    ix = S.sfc_index_build(dev(g0), dev(m0), K=7, curves=2, dims=4, bits=10, window=8, pca_sample=0)
    ex0 = S.sfc_index_export(ix)
    ix.close()
    g = np.full((160, 160, 3), 0.25, np.float32)
    m = np.ones((160, 160), np.uint8)
    m[70:90, 70:90] = 0
    ex = check_all_modes(S, g, m, K=7, curves=2, dims=4, bits=10, window=8, basis=ex0["basis"], mean=ex0["mean"])
    assert np.all(ex["keys"] == ex["keys"][:, :1])
    assert np.array_equal(ex["sids"], np.tile(np.arange(len(ex["dict"]), dtype=np.uint32), (2, 1)))


def test_sort_at_the_sample_sort_limit(S):
    # 2^20 dictionary entries take the sample sort, more the LSD sort; both give
    # the oracle's sort (grey noise images, every patch known, K = 7)
    for X, Y in ((1030, 1030), (1031, 1030)):
        g = np.random.default_rng(X).random((Y, X, 1)).astype(np.float32)
        m = np.ones((Y, X), np.uint8)
        ix = S.sfc_index_build(dev(g), dev(m), K=7, curves=1, dims=4, bits=12, window=8, pca_sample=4096,
                               keep_intermediates=1)
        ex = S.sfc_index_export(ix, proj=True)
        ix.close()
        assert len(ex["dict"]) == (X - 6) * (Y - 6)
        sk, si = O.sort(ex["keys"][0])
        assert np.array_equal(sk, ex["skeys"][0]) and np.array_equal(si, ex["sids"][0])
    assert S.sfc_status() == 0
