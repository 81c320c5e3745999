"""Stored indices (sfc_index_save / sfc_index_load) and queries from another
grid (sfc_query_batch_dict), through the C-ABI (needs a GB300).

Bars: a loaded index exports the same arrays and answers queries with the
same candidates, picks and costs (bit-identical) as the one saved; queries
from another grid match the oracle's query with the two grids (picks equal,
costs within 1e-5 of its exact cost); a corrupt or truncated file is refused.
"""
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_06326_gb300 import synth

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-5


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


@pytest.mark.parametrize("kw", [dict(), dict(knn=16), dict(curve=1), dict(cost=1), dict(select=1, shifts="rand")])
def test_save_load_round_trip(S, tmp_path, kw):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)
    t = np.concatenate([synth.front_targets(m, 7, cap=40, cfg=2), synth.random_targets(m, 7, 10, cfg=2)])
    kw = dict(kw)
    if kw.get("shifts") == "rand":
        kw["shifts"] = np.random.default_rng(2).integers(0, 1 << 10, (8, 6)).astype(np.int32)
    ix = S.sfc_index_build(dev(g), dev(m), K=7, curves=8, dims=6, bits=12, window=16, pca_sample=0, **kw)
    path = str(tmp_path / "ix.sfc")
    S.sfc_index_save(ix, path)
    assert os.path.getsize(path) > 8 * ix.N * 12
    iy = S.sfc_index_load(path)
    assert (iy.N, iy.m, iy.s) == (ix.N, ix.m, ix.s)
    for k in ("K", "curves", "dims", "bits", "window", "select", "knn", "curve", "cost"):
        assert getattr(iy.params, k) == getattr(ix.params, k), k
    ea, eb = S.sfc_index_export(ix), S.sfc_index_export(iy)
    for k in ea:
        assert np.array_equal(ea[k], eb[k], equal_nan=True), k
    outs = []
    for h in (ix, iy):
        _, _, cand, nc = S.sfc_query_candidates(h, dev(g), dev(m), dev(t))
        pk, cs = S.sfc_query_batch(h, dev(g), dev(m), dev(t))
        outs.append((cand.cpu().numpy(), nc.cpu().numpy(), pk.cpu().numpy(), cs.cpu().numpy()))
    for a, b in zip(*outs):
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    assert S.sfc_status() == 0
    ix.close()
    iy.close()


def test_query_from_another_grid_matches_oracle(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)      # the dictionary's image
    g2, m2 = synth.voronoi2d(80, cfg=2, seed_sub=11)   # another image, another size
    K, C_, D, bits, W = 7, 8, 6, 12, 24
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0)
    ex = S.sfc_index_export(ix)
    oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
    t = np.concatenate([synth.front_targets(m2, K, cap=40, cfg=2), synth.random_targets(m2, K, 10, cfg=2)])
    pk, cs = S.sfc_query_batch_dict(ix, dev(g), dev(g2), dev(m2), dev(t))
    pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
    for i, tl in enumerate(O.centres_to_lin(t, O.geometry(g2)[1])):
        r = O.query_dict(oix, g, g2, m2, tl, W)
        assert pk[i] == r["pick"]
        assert abs(float(cs[i]) - r["cost"]) <= COST_RTOL * r["cost"] and (cs[i] == 0) == (r["cost"] == 0)
    # the same grid on both sides is sfc_query_batch, bit for bit
    t1 = synth.front_targets(m, K, cap=30, cfg=2)
    a = S.sfc_query_batch_dict(ix, dev(g), dev(g), dev(m), dev(t1))
    b = S.sfc_query_batch(ix, dev(g), dev(m), dev(t1))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))
    assert S.sfc_status() == 0
    ix.close()


def test_query_from_a_loaded_index_and_3d(S, tmp_path):
    g, m = synth.spheres3d(24, block=4, missing=0.1, seed_sub=1)
    g2, m2 = synth.spheres3d(20, block=4, missing=0.15, seed_sub=2)
    K, C_, D, bits, W = 5, 4, 8, 16, 32
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0)
    ex = S.sfc_index_export(ix)
    path = str(tmp_path / "v.sfc")
    S.sfc_index_save(ix, path)
    ix.close()
    iy = S.sfc_index_load(path)
    oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
    t = synth.front_targets(m2, K, cap=30, cfg=3)
    pk, cs = S.sfc_query_batch_dict(iy, dev(g), dev(g2), dev(m2), dev(t))
    pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
    for i, tl in enumerate(O.centres_to_lin(t, O.geometry(g2)[1])):
        r = O.query_dict(oix, g, g2, m2, tl, W)
        assert pk[i] == r["pick"] and abs(float(cs[i]) - r["cost"]) <= COST_RTOL * r["cost"]
    assert S.sfc_status() == 0
    iy.close()


def test_bad_files_and_grids_are_refused(S, tmp_path):
    g, m = synth.sines2d(64)
    ix = S.sfc_index_build(dev(g), dev(m), K=9, curves=2, dims=4, bits=8, window=8)
    path = tmp_path / "i.sfc"
    S.sfc_index_save(ix, str(path))
    raw = path.read_bytes()
    (tmp_path / "trunc.sfc").write_bytes(raw[: len(raw) // 2])
    (tmp_path / "junk.sfc").write_bytes(b"not an index" * 10)
    for bad in ("trunc.sfc", "junk.sfc", "missing.sfc"):
        with pytest.raises(RuntimeError):
            S.sfc_index_load(str(tmp_path / bad))
    rgb = np.zeros((32, 32, 3), np.float32)
    with pytest.raises(RuntimeError, match="channel"):
        S.sfc_query_batch_dict(ix, dev(g), dev(rgb), dev(np.ones((32, 32), np.uint8)),
                               dev(np.array([[10, 10]], np.int32)))
    assert S.sfc_status() == 0
    ix.close()
