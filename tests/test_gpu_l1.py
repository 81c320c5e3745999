"""The L1 cost (Sec. III.K, cost = SFC_COST_L1) vs the oracle, through the
C-ABI (needs a GB300).

Bars as for L2: picks equal, reported FP32 costs within 1e-5 of the oracle's
exact FP64 cost, candidate sets bit-exact, the fill loop's log and output
bit-identical.
"""
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


def close(gpu, exact):
    gpu = np.asarray(gpu, np.float64)
    exact = np.asarray(exact, np.float64)
    return np.all(np.abs(gpu - exact) <= COST_RTOL * np.abs(exact)) and np.all((gpu == 0) == (exact == 0))


def check_fullscan_l1(S, g, m, t, K, w=None):
    fp, fc = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=K, ch_weights=w, norm=S.SFC_COST_L1)
    d = O.dict_extract(m, K)
    op, oc = O.fullscan(g, m, K, d, O.centres_to_lin(t, O.geometry(g)[1]), w, norm=1)
    assert np.array_equal(fp.cpu().numpy(), op)
    assert close(fc.cpu().numpy(), oc)
    # the L1 picks are not the L2 picks in general
    lp, _ = O.fullscan(g, m, K, d, O.centres_to_lin(t, O.geometry(g)[1]), w)
    return op, lp


def test_l1_fullscan_sines(S):
    g, m = synth.sines2d(128)
    op, lp = check_fullscan_l1(S, g, m, synth.front_targets(m, 9), 9)
    assert not np.array_equal(op, lp)


def test_l1_fullscan_rgb_weighted_and_random(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=2)
    t = np.concatenate([synth.front_targets(m, 7, cap=40, cfg=2), synth.random_targets(m, 7, 20, cfg=2)])
    check_fullscan_l1(S, g, m, t, 7)
    check_fullscan_l1(S, g, m, t, 7, w=np.array([1.0, 2.0, 0.5], np.float32))


def test_l1_fullscan_ties_and_3d(S):
    rng = np.random.default_rng(5)
    g = rng.random((40, 40, 1)).astype(np.float32)
    g[30:35, 30:35] = g[3:8, 3:8]
    m = np.ones((40, 40), np.uint8)
    op, _ = check_fullscan_l1(S, g, m, np.array([[32, 32], [5, 5]], np.int32), 5)
    assert O.dict_extract(m, 5)[op[0]] == 5 * 40 + 5
    g3, m3 = synth.spheres3d(24, block=4, missing=0.1)
    check_fullscan_l1(S, g3, m3, synth.front_targets(m3, 5, cap=30, cfg=3), 5)


def test_l1_tensor_prescore_rejected(S):
    g, m = synth.sines2d(64)
    t = synth.front_targets(m, 9, cap=20)
    with pytest.raises(RuntimeError, match="L2"):
        S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=9, precision=S.SFC_FP16, norm=S.SFC_COST_L1)
    assert S.sfc_status() == 0


@pytest.mark.parametrize("knn", [0, 40])
def test_l1_sfc_queries(S, knn):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)
    K, C_, D, bits, W = 7, 8, 6, 12, 16
    t = np.concatenate([synth.front_targets(m, K, cap=40, cfg=2), synth.random_targets(m, K, 10, cfg=2)])
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0, knn=knn,
                           cost=S.SFC_COST_L1)
    ex = S.sfc_index_export(ix)
    oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
    _, _, cand, ncand = S.sfc_query_candidates(ix, dev(g), dev(m), dev(t))
    pk, cs = S.sfc_query_batch(ix, dev(g), dev(m), dev(t))
    cand, ncand, pk, cs = cand.cpu().numpy(), ncand.cpu().numpy(), pk.cpu().numpy(), cs.cpu().numpy()
    for i, tl in enumerate(O.centres_to_lin(t, O.geometry(g)[1])):
        r = O.query_knn(oix, g, m, tl, knn, norm=1) if knn else O.query(oix, g, m, tl, W, norm=1)
        assert np.array_equal(cand[i, :ncand[i]], r["cand"])
        assert pk[i] == r["pick"] and close(cs[i], r["cost"])
    assert S.sfc_status() == 0
    ix.close()


def test_l1_fill_fullscan_bit_identical(S):
    g, m = synth.sines2d(128)
    og, om, olog, osteps = O.inpaint(g, m, 9, mode=0, prio=0, norm=1)
    gd, md = dev(g), dev(m)
    steps, log = S.inpaint_run(gd, md, mode=S.SFC_MODE_FULLSCAN, K=9, priority=0, cost=S.SFC_COST_L1)
    assert steps == osteps and np.array_equal(log.cpu().numpy(), olog)
    assert np.array_equal(gd.cpu().numpy(), og) and md.cpu().numpy().all()
    # a different fill than the L2 one
    _, _, llog, _ = O.inpaint(g, m, 9, mode=0, prio=0)
    assert not np.array_equal(llog, olog)
