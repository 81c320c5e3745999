"""The split form of small query batches (needs a GB300): batches of up to 32
queries spread each query's rescore over many CTAs (the fill loop asks one
query per step).  The FP32 cost of every candidate is computed with the same
operations in the same order as in the one-CTA form, so the bar is bit
equality: picks and cost bits of the split form (batches of 1, 5 and 32)
equal those of the one-CTA form (the whole batch of more than 32 queries in
one launch), for the window search, the k-NN lists, channel weights, the L1
cost, a 3-D volume, targets on another grid, and invalid centres; the picks
also equal the oracle's (Fig. 1(b)-(d))."""
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


def split_vs_whole(run, t, sizes=(1, 5, 32)):
    """run(centres) -> (pick, cost); the whole batch (> 32: one CTA per query)
    against batches of each size (the split form)."""
    assert len(t) > 32
    wp, wc = run(t)
    for b in sizes:
        parts = [run(t[i:i + b]) for i in range(0, len(t), b)]
        sp = torch.cat([p for p, _ in parts])
        sc = torch.cat([c for _, c in parts])
        assert torch.equal(sp, wp), b
        assert torch.equal(sc.view(torch.int32), wc.view(torch.int32)), b
    return wp, wc


def test_split_window_search_equals_one_cta_and_oracle(S):
    g, m = synth.voronoi2d(128, cfg=2, seed_sub=21)
    t = np.concatenate([synth.front_targets(m, 9, cap=60, cfg=2), synth.random_targets(m, 9, 20, cfg=2)])
    K, C_, D, bits, W = 9, 8, 6, 12, 32
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0)
    wp, _ = split_vs_whole(lambda c: S.sfc_query_batch(ix, dev(g), dev(m), dev(c)), t)
    ex = S.sfc_index_export(ix)
    oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
    lin = O.centres_to_lin(t, O.geometry(g)[1])
    wp = wp.cpu().numpy()
    for i in range(0, len(t), 7):
        assert wp[i] == O.query(oix, g, m, lin[i], W)["pick"]
    assert S.sfc_status() == 0
    ix.close()


@pytest.mark.parametrize("kw", [dict(knn=24), dict(ch_weights=np.array([1.0, 2.0, 0.5], np.float32)),
                                dict(cost=1), dict(select=1)])
def test_split_variants(S, kw):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=22)
    t = np.concatenate([synth.front_targets(m, 7, cap=40, cfg=2), synth.random_targets(m, 7, 10, cfg=2)])
    params = dict(K=7, curves=4, dims=6, bits=10, window=24, pca_sample=0)
    if kw.get("cost") == 1:
        kw = dict(cost=S.SFC_COST_L1)
    if kw.get("select") == 1:
        kw = dict(select=S.SFC_SELECT_BEST)
    ix = S.sfc_index_build(dev(g), dev(m), **params, **kw)
    split_vs_whole(lambda c: S.sfc_query_batch(ix, dev(g), dev(m), dev(c)), t)
    assert S.sfc_status() == 0
    ix.close()


def test_split_3d_and_another_grid(S):
    g, m = synth.spheres3d(24, block=4, missing=0.1, seed_sub=5)
    t = synth.front_targets(m, 5, cap=48, cfg=3)
    ix = S.sfc_index_build(dev(g), dev(m), K=5, curves=4, dims=8, bits=16, window=32, pca_sample=0)
    split_vs_whole(lambda c: S.sfc_query_batch(ix, dev(g), dev(m), dev(c)), t)
    ix.close()
    g1, m1 = synth.voronoi2d(96, cfg=2, seed_sub=23)
    g2, m2 = synth.voronoi2d(80, cfg=2, seed_sub=24)
    ix = S.sfc_index_build(dev(g1), dev(m1), K=7, curves=8, dims=6, bits=12, window=24, pca_sample=0)
    t2 = np.concatenate([synth.front_targets(m2, 7, cap=40, cfg=2), synth.random_targets(m2, 7, 10, cfg=2)])
    split_vs_whole(lambda c: S.sfc_query_batch_dict(ix, dev(g1), dev(g2), dev(m2), dev(c)), t2)
    assert S.sfc_status() == 0
    ix.close()


def test_split_invalid_centre(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=25)
    t = synth.front_targets(m, 7, cap=40, cfg=2)
    t = np.concatenate([t[:3], np.array([[0, 0]], np.int32), t[3:]])  # the patch leaves the grid
    ix = S.sfc_index_build(dev(g), dev(m), K=7, curves=4, dims=6, bits=10, window=24, pca_sample=0)
    wp, wc = S.sfc_query_batch(ix, dev(g), dev(m), dev(t))
    assert S.sfc_status() == S.SFC_EDEVICE
    sp, sc = S.sfc_query_batch(ix, dev(g), dev(m), dev(t[:5]))
    assert S.sfc_status() == S.SFC_EDEVICE
    assert sp[3].item() == -1 and np.isnan(sc[3].item())
    assert torch.equal(sp, wp[:5]) and torch.equal(sc.view(torch.int32), wc[:5].view(torch.int32))
    one = S.sfc_query_batch(ix, dev(g), dev(m), dev(t[3:4]))
    assert S.sfc_status() == S.SFC_EDEVICE
    assert one[0].item() == -1 and np.isnan(one[1].item())
    assert S.sfc_status() == 0
    ix.close()
