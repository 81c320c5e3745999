"""Tile shapes of the FP32 full scan and their tuner (needs a GB300): every
compiled (queries per tile, entries per thread) shape gives the same picks and
cost bits (the exact full scan of Sec. I), equal to the oracle's picks, for the
L2 and L1 costs, channel weights, a query count below the tile and an invalid
centre; sfc_tune_tiles times every shape, keeps the fastest and reports the
table."""
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
    sfc.sfc_tile_shape(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


NSHAPES = 7


def test_every_shape_gives_the_same_scan(S):
    g, m = synth.voronoi2d(128, cfg=2, seed_sub=61)
    t = np.concatenate([synth.front_targets(m, 7, cap=40, cfg=2), synth.random_targets(m, 7, 13, cfg=2)])
    w = np.array([1.0, 2.0, 0.5], np.float32)
    for kw in (dict(), dict(ch_weights=w), dict(norm=S.SFC_COST_L1)):
        for tt in (t, t[:3]):  # fewer queries than a tile
            ref = None
            for k in range(NSHAPES):
                assert S.sfc_tile_shape(k) == k
                p, c = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(tt), K=7, **kw)
                if ref is None:
                    ref = (p, c)
                else:
                    assert torch.equal(p, ref[0]) and torch.equal(c.view(torch.int32), ref[1].view(torch.int32)), k
    op, _ = O.fullscan(g, m, 7, O.dict_extract(m, 7), O.centres_to_lin(t, O.geometry(g)[1]))
    S.sfc_tile_shape(3)
    p, _ = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=7)
    assert np.array_equal(p.cpu().numpy(), op)
    bad = np.concatenate([t[:5], np.array([[0, 0]], np.int32)])
    p, c = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(bad), K=7)
    assert S.sfc_status() == S.SFC_EDEVICE
    assert p[-1].item() == -1 and np.isnan(c[-1].item())
    S.sfc_tile_shape(0)
    assert S.sfc_status() == 0


def test_tuner_keeps_the_fastest(S):
    g, m = synth.voronoi2d(160, cfg=2, seed_sub=62)
    t = synth.front_targets(m, 9, cap=64, cfg=2)
    table, chosen = S.sfc_tune_tiles(dev(g), dev(m), dev(m), dev(t), reps=2, K=9)
    assert table.shape == (NSHAPES, 3)
    assert [tuple(r[:2]) for r in table] == [(8, 4), (8, 2), (16, 2), (4, 4), (4, 8), (16, 4), (32, 2)]
    assert np.all(table[:, 2] > 0)
    assert chosen == int(np.argmin(table[:, 2]))
    assert S.sfc_tile_shape(-1) == chosen
    with pytest.raises(RuntimeError):
        S.sfc_tune_tiles(dev(g), dev(m), dev(m), dev(t), reps=1, K=9, precision=S.SFC_FP16)
    assert S.sfc_tile_shape(-1) == chosen  # a refused call changes nothing
    S.sfc_tile_shape(0)
    assert S.sfc_status() == 0
