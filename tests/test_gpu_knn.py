"""SFC queries with the paper's exact k-NN lists (Sec. II.D, knn = k) vs the
oracle, through the C-ABI (needs a GB300).

Bars: candidate sets bit-exact -- the sorted union over the selected indices
of the k nearest dictionary entries in the quantised principal space (ties by
id), which the oracle finds by brute force over every entry; picks equal and
costs within 1e-5 of the oracle's exact cost.  The oracle is rebuilt from the
GPU's exported basis (the checkpoint split: keys, quantised coordinates and
lists are then exact).
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


def run_case(S, g, m, t, K, C_, D, bits, k, select=0, shifts=None, cur=None):
    cur = m if cur is None else cur
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=16, pca_sample=0, knn=k,
                           select=select, shifts=shifts)
    ex = S.sfc_index_export(ix)
    oix = O.build_index(g, m, K, C_, D, bits, shifts=shifts, basis=ex["basis"], mean=ex["mean"])
    assert np.array_equal(oix["skeys"], ex["skeys"]) and np.array_equal(oix["sids"], ex["sids"])
    qk, pos, cand, ncand = S.sfc_query_candidates(ix, dev(g), dev(cur), dev(t))
    pk, cs = S.sfc_query_batch(ix, dev(g), dev(cur), dev(t))
    cand, ncand = cand.cpu().numpy(), ncand.cpu().numpy()
    pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
    lin = O.centres_to_lin(t, O.geometry(g)[1])
    for i, tl in enumerate(lin):
        r = O.query_knn(oix, g, cur, tl, k, select=select)
        assert np.array_equal(cand[i, :ncand[i]], r["cand"]), f"candidate set of query {i}"
        assert pk[i] == r["pick"]
        assert abs(float(cs[i]) - r["cost"]) <= COST_RTOL * r["cost"] and (cs[i] == 0) == (r["cost"] == 0)
    assert S.sfc_status() == 0
    ix.close()
    return oix


def test_knn_rgb_front_and_random_targets(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)
    t = np.concatenate([synth.front_targets(m, 7, cap=60, cfg=2), synth.random_targets(m, 7, 20, cfg=2)])
    oix = run_case(S, g, m, t, 7, 8, 6, 12, 24)
    assert oix["N"] > 48 * 8  # the lists come from the box scan, not only the first window


@pytest.mark.parametrize("k", [1, 33, 80, 128])
def test_knn_list_lengths(S, k):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=4)
    t = synth.front_targets(m, 7, cap=30, cfg=2)
    run_case(S, g, m, t, 7, 4, 8, 16, k)


def test_knn_select_best_and_shifts(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=5)
    t = synth.front_targets(m, 7, cap=40, cfg=2)
    rng = np.random.default_rng(9)
    sh = rng.integers(0, 1 << 10, (8, 6)).astype(np.int32)
    run_case(S, g, m, t, 7, 8, 6, 10, 20, select=1, shifts=sh)
    run_case(S, g, m, t, 7, 8, 6, 10, 20, select=0, shifts=sh)


def test_knn_partly_filled_mask(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=6)
    cur = m.copy()
    cur[40:56, 40:56] = 0  # more unknown pixels at query time than at build time
    t = np.concatenate([synth.front_targets(cur, 7, cap=40, cfg=2), synth.random_targets(cur, 7, 10, cfg=2)])
    run_case(S, g, m, t, 7, 8, 6, 12, 16, cur=cur)


def test_knn_covering_dictionary_equals_fullscan(S):
    g, m = synth.sines2d(24)
    t = synth.front_targets(m, 9, cap=30)
    N = len(O.dict_extract(m, 9))
    assert N == 112  # k = 128 > N: every list is the whole dictionary
    oix = run_case(S, g, m, t, 9, 2, 4, 8, 128)
    fp, _ = O.fullscan(g, m, 9, oix["dict"], O.centres_to_lin(t, O.geometry(g)[1]))
    r = [O.query_knn(oix, g, m, tl, 128)["pick"] for tl in O.centres_to_lin(t, O.geometry(g)[1])]
    assert np.array_equal(fp, r)


def test_knn_3d_truncated_keys(S):
    g, m = synth.spheres3d(32, block=4, missing=0.1)
    t = synth.front_targets(m, 5, cap=40, cfg=3)
    # D * b = 12 * 21 = 252 bits: keys keep the top 64 (dims 0-3 six bits, 4-11 five)
    run_case(S, g, m, t, 5, 4, 12, 21, 40)


def test_knn_ties_and_constant_grid(S):
    g = np.full((40, 40, 2), 0.25, np.float32)
    m = np.ones((40, 40), np.uint8)
    m[10:14, 10:14] = 0
    t = np.array([[12, 9], [3, 3], [36, 36]], np.int32)
    run_case(S, g, m, t, 3, 2, 2, 8, 7)  # all coordinates equal: the lists are the lowest ids


def test_knn_deep_recursion_256(S):
    """N ~ 55k: regions split many levels below the root before the leaf scans
    (leaves hold at most 2,048 slots)."""
    g, m = synth.voronoi2d(256, cfg=2, seed_sub=8)
    t = np.concatenate([synth.front_targets(m, 9, cap=24, cfg=2), synth.random_targets(m, 9, 8, cfg=2)])
    oix = run_case(S, g, m, t, 9, 8, 8, 16, 80)
    assert oix["N"] > 40_000


def principal_sin_max(B1, B2):
    """sin of the largest principal angle between the column spaces of B1 and B2."""
    Q1 = np.linalg.qr(np.asarray(B1, np.float64))[0]
    Q2 = np.linalg.qr(np.asarray(B2, np.float64))[0]
    return np.linalg.norm(Q2 - Q1 @ (Q1.T @ Q2), 2)


@pytest.mark.parametrize("priority", [0, 1])
def test_fill_with_the_papers_defaults_bit_identical(S, priority):
    # the fill loop of Sec. I run with the settings of the paper's evaluation
    # (Sec. III: K = 9, D = 10, k = 80 nearest per index, c = 0.6, byte
    # coordinates) on the 128^2 grey image with its 24^2 hole: every step's
    # (target, pick) and the filled image equal the oracle's
    g, m = synth.sines2d(128)
    K, C_, D, bits, k = 9, 8, 10, 8, 80
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=16, pca_sample=0, knn=k)
    ex = S.sfc_index_export(ix)
    ix.close()
    assert S.sfc_status() == 0
    # the image's noise leaves a flat tail of eigenvalues (l_11 / l_10 ~ 0.99):
    # the basis is still the oracle's -- eigenvalues within 1e-10 relative and
    # every principal angle between the D-dimensional subspaces below 1e-6
    d = ex["dict"]
    for cv in range(C_):
        B, mu, ev, cov = O.pca(g, K, d, ex["subsets"][cv], 0, D)
        assert np.allclose(ex["evals"][cv][:D], ev[:D], rtol=1e-10, atol=0)
        assert principal_sin_max(ex["basis"][cv], B) < 1e-6
    oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
    og, om, olog, osteps = O.inpaint(g, m, K, mode=1, prio=priority, ix=oix, knn=k)
    gd, md = dev(g), dev(m)
    steps, log = S.inpaint_run(gd, md, mode=S.SFC_MODE_SFC, K=K, curves=C_, dims=D, bits=bits, window=16, knn=k,
                               basis=ex["basis"], mean=ex["mean"], priority=priority)
    assert steps == osteps and np.array_equal(log.cpu().numpy(), olog)
    assert np.array_equal(gd.cpu().numpy(), og) and md.cpu().numpy().all()
    assert S.sfc_status() == 0
