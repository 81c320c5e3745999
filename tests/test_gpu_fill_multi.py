"""The inpainting loop of several images at once (inpaint_run_multi, SFC mode;
needs a GB300).  Each image must end exactly as its own inpaint_run leaves it
(the loop of Sec. I / Fig. 1(a), one step per round for every image): the same
grid bits, mask, log and step count -- for images of different sizes, the
confidence and the Criminisi priorities, a step cap, an image with nothing to
fill, 3-D volumes, and, from an imported basis, the oracle's loop itself."""
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


def one_by_one(S, images, max_steps=0, **params):
    out = []
    for g, m in images:
        gd, md = dev(g), dev(m)
        n, log = S.inpaint_run(gd, md, mode=S.SFC_MODE_SFC, max_steps=max_steps, **params)
        out.append((gd.cpu().numpy(), md.cpu().numpy(), log.cpu().numpy(), n))
    return out


def all_at_once(S, images, max_steps=0, **params):
    gds = [dev(g) for g, _ in images]
    mds = [dev(m) for _, m in images]
    steps, logs = S.inpaint_run_multi(gds, mds, max_steps=max_steps, **params)
    return [(gd.cpu().numpy(), md.cpu().numpy(), lg.cpu().numpy(), n) for gd, md, lg, n in zip(gds, mds, logs, steps)]


def check_same(a, b):
    assert len(a) == len(b)
    for i, ((g1, m1, l1, n1), (g2, m2, l2, n2)) in enumerate(zip(a, b)):
        assert n1 == n2, i
        assert np.array_equal(l1, l2), i
        assert np.array_equal(m1, m2), i
        assert np.array_equal(g1.view(np.uint32), g2.view(np.uint32)), i


def test_multi_images_of_different_sizes(S):
    images = [synth.voronoi2d(96, cfg=2, seed_sub=41), synth.voronoi2d(64, cfg=2, seed_sub=42),
              synth.voronoi2d(128, 80, cfg=2, seed_sub=43)]
    params = dict(K=7, curves=4, dims=6, bits=12, window=24, pca_sample=0)
    ref = one_by_one(S, images, **params)
    got = all_at_once(S, images, **params)
    check_same(ref, got)
    assert all(m.all() for _, m, _, _ in got)
    assert S.sfc_status() == 0


def test_multi_criminisi_step_cap_and_a_full_image(S):
    g0, m0 = synth.voronoi2d(80, cfg=2, seed_sub=44)
    g1, m1 = synth.voronoi2d(72, cfg=2, seed_sub=45)
    full = (g1.copy(), np.ones_like(m1))  # nothing to fill: done at the first round
    images = [(g0, m0), full, (g1, m1)]
    params = dict(K=5, curves=8, dims=5, bits=10, window=12, pca_sample=0, priority=1)
    for cap in (0, 7):
        ref = one_by_one(S, images, max_steps=cap, **params)
        got = all_at_once(S, images, max_steps=cap, **params)
        check_same(ref, got)
        assert got[1][3] == 0
        if cap:
            assert got[0][3] == cap and got[2][3] == cap
    assert S.sfc_status() == 0


def test_multi_more_images_than_the_split_form_takes(S):
    # 36 images: each round's search is the one-CTA multi-image launch
    images = [synth.voronoi2d(40 + 4 * (i % 5), cfg=2, seed_sub=60 + i) for i in range(36)]
    params = dict(K=5, curves=4, dims=4, bits=10, window=8, pca_sample=0)
    ref = one_by_one(S, images, max_steps=25, **params)
    got = all_at_once(S, images, max_steps=25, **params)
    check_same(ref, got)
    assert S.sfc_status() == 0


def test_multi_3d(S):
    images = [synth.spheres3d(20, block=4, missing=0.05, seed_sub=46),
              synth.spheres3d(24, block=4, missing=0.05, seed_sub=47)]
    params = dict(K=3, curves=4, dims=6, bits=12, window=16, pca_sample=0)
    ref = one_by_one(S, images, max_steps=60, **params)
    got = all_at_once(S, images, max_steps=60, **params)
    check_same(ref, got)
    assert S.sfc_status() == 0


def test_multi_matches_the_oracle_loop(S):
    # a shared imported basis: the oracle's index of each image from the same basis
    g0, m0 = synth.voronoi2d(64, cfg=2, seed_sub=48)
    g1, m1 = synth.voronoi2d(56, cfg=2, seed_sub=49)
    K, C_, D, bits, W = 5, 8, 5, 10, 12
    ix = S.sfc_index_build(dev(g0), dev(m0), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0)
    ex = S.sfc_index_export(ix)
    ix.close()
    got = all_at_once(S, [(g0, m0), (g1, m1)], K=K, curves=C_, dims=D, bits=bits, window=W,
                      basis=ex["basis"], mean=ex["mean"], priority=1)
    for (g, m), (gg, gm, glog, gsteps) in zip([(g0, m0), (g1, m1)], got):
        oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
        og, om, olog, osteps = O.inpaint(g, m, K, mode=1, prio=1, ix=oix, W=W)
        assert gsteps == osteps and np.array_equal(glog, olog)
        assert np.array_equal(gg, og) and np.array_equal(gm, om)
    assert S.sfc_status() == 0


def test_multi_refusals(S):
    g, m = synth.voronoi2d(48, cfg=2, seed_sub=50)
    with pytest.raises(RuntimeError):
        S.inpaint_run_multi([dev(g)], [dev(m)], K=5, curves=4, dims=4, window=8, pca_sample=0, knn=8)
    g3, m3 = synth.spheres3d(16, block=4, missing=0.05)
    with pytest.raises(RuntimeError):  # another dimension than image 0
        S.inpaint_run_multi([dev(g), dev(g3)], [dev(m), dev(m3)], K=3, curves=4, dims=4, window=8, pca_sample=0)
