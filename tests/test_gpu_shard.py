"""The dictionary split of the full scan on the GPU (needs a GB300): S shards
of one scan run one after another on this GPU (each rank of a multi-GPU run
does one of them), the exchange steps done here on the host as the collectives
would do them (element-wise minimum of the shard minima, then the (FP64 cost,
id) minimum over the shards' band results).  Bars: picks and costs equal
fullscan_query_batch's bit for bit for every shard count, including ties across
shards, weights, the L1 cost, 3-D grids, invalid centres and shards with no
entries; query sharding over one index answers like the whole batch."""
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


def split_on_one_gpu(g, m, t, K, nshards, **params):
    from paper_1712_06326_gb300 import shard as SH

    shards = [SH.Shard(dev(g), dev(m), dev(m), dev(t), K, s, nshards, **params) for s in range(nshards)]
    assert shards[0].j0 == 0 and shards[-1].j1 == shards[0].N
    assert all(a.j1 == b.j0 for a, b in zip(shards, shards[1:]))
    mins = torch.stack([sh.scan() for sh in shards])
    gmin = mins.min(dim=0).values.contiguous()  # the all-reduce-min
    parts = [sh.band(gmin) for sh in shards]    # every rank's band result
    pick, cost = SH.merge_shard_results(*(torch.stack([p[i] for p in parts]) for i in range(3)))
    for sh in shards:
        sh.close()
    return pick, cost


@pytest.mark.parametrize("nshards", [1, 2, 3, 7])
def test_split_equals_single_gpu_scan(S, nshards):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)
    t = np.concatenate([synth.front_targets(m, 7, cap=40, cfg=2), synth.random_targets(m, 7, 24, cfg=2)])
    g[60:67, 70:77] = g[3:10, 3:10]  # an exact duplicate far from the original: a tie across shards
    t = np.concatenate([t, np.array([[6, 6], [73, 63]], np.int32)])
    w = np.array([1.0, 2.0, 0.5], np.float32)
    for kw in (dict(), dict(ch_weights=w), dict(cost=S.SFC_COST_L1)):
        fp, fc = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=7,
                                        ch_weights=kw.get("ch_weights"), norm=kw.get("cost", 0))
        sp, sc = split_on_one_gpu(g, m, t, 7, nshards, **kw)
        assert torch.equal(sp, fp) and torch.equal(sc.view(torch.int32), fc.view(torch.int32))
    op, _ = O.fullscan(g, m, 7, O.dict_extract(m, 7), O.centres_to_lin(t, O.geometry(g)[1]))
    sp, _ = split_on_one_gpu(g, m, t, 7, nshards)
    assert np.array_equal(sp.cpu().numpy(), op)
    assert S.sfc_status() == 0


def test_split_3d_invalid_centres_and_empty_shards(S):
    g, m = synth.spheres3d(24, block=4, missing=0.1)
    t = synth.front_targets(m, 5, cap=30, cfg=3)
    t = np.concatenate([t, np.array([[0, 0, 0]], np.int32)])  # invalid: the patch leaves the grid
    fp, fc = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=5)
    assert S.sfc_status() == S.SFC_EDEVICE
    sp, sc = split_on_one_gpu(g, m, t, 5, 4)
    assert S.sfc_status() == S.SFC_EDEVICE
    assert torch.equal(sp, fp) and sp[-1].item() == -1 and np.isnan(sc[-1].item())
    assert torch.equal(sc[:-1].view(torch.int32), fc[:-1].view(torch.int32))
    # more shards than dictionary entries: most shards are empty
    g2 = np.random.default_rng(4).random((10, 10, 1)).astype(np.float32)
    m2 = np.zeros((10, 10), np.uint8)
    m2[0:3, 0:5] = 1  # three fully known 3x3 patches
    t2 = np.array([[5, 5], [1, 1], [3, 1]], np.int32)
    fp2, fc2 = S.fullscan_query_batch(dev(g2), dev(m2), dev(m2), dev(t2), K=3)
    sp2, sc2 = split_on_one_gpu(g2, m2, t2, 3, 6)
    assert torch.equal(sp2, fp2) and torch.equal(sc2.view(torch.int32), fc2.view(torch.int32))
    assert S.sfc_status() == 0


def test_query_sharding_equals_whole_batch(S):
    from paper_1712_06326_gb300 import shard as SH

    g, m = synth.voronoi2d(128, cfg=2, seed_sub=6)
    t = synth.front_targets(m, 9, cap=100, cfg=2)
    ix = S.sfc_index_build(dev(g), dev(m), K=9, curves=8, dims=6, bits=12, window=32, pca_sample=0)
    wp, wc = S.sfc_query_batch(ix, dev(g), dev(m), dev(t))
    for world in (2, 3, 8):
        parts = [SH.shard_bounds(len(t), r, world) for r in range(world)]
        got = [S.sfc_query_batch(ix, dev(g), dev(m), dev(t[a:b])) for a, b in parts]
        assert torch.equal(torch.cat([p for p, _ in got]), wp)
        assert torch.equal(torch.cat([c for _, c in got]).view(torch.int32), wc.view(torch.int32))
    # the single-process path of the module (world 1) is the plain batch
    sp, sc = SH.query_batch_split(ix, dev(g), dev(m), dev(t))
    assert torch.equal(sp, wp)
    ix.close()
    assert S.sfc_status() == 0
