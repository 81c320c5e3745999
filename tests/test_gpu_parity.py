"""CUDA path vs the CPU oracle, through the C-ABI (needs a GB300).

Bars: dictionary ids, subsets, projections (FP32 chain), lo/scale, keys, sorted
orders, query keys, positions and candidate sets bit-exact; picks equal; the
reported cost (the FP32 cost of the pick) within COST_RTOL of the oracle's exact
FP64 cost; the PCA basis (another summation order and eigen-solver) within the
tolerances stated below; the fill loop's log and output bit-identical.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_06326_gb300 import synth

pytestmark = pytest.mark.gpu

# FP32 cost vs exact cost: the target's bar (1e-5 relative); zero stays zero
COST_RTOL = 1e-5


def cost_close(gpu, exact):
    gpu = np.asarray(gpu, np.float64)
    exact = np.asarray(exact, np.float64)
    return np.all(np.abs(gpu - exact) <= COST_RTOL * np.abs(exact)) and np.all((gpu == 0) == (exact == 0))


@pytest.fixture(scope="module")
def S():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1712_06326_gb300 import sfc

    torch.cuda.set_device(0)
    return sfc


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ext_of(g):
    return O.geometry(g)[1]


def oracle_ix(ex, grid, K, C_, D, bits, shifts=None):
    ndim, ext, ch = O.geometry(grid)
    return dict(ndim=ndim, ext=ext, ch=ch, K=K, C=C_, D=D, bits=bits, dict=ex["dict"], N=len(ex["dict"]),
                subset=np.ascontiguousarray(ex["subsets"]), m=ex["subsets"].shape[1], basis=ex["basis"],
                mean=ex["mean"], lo=ex["lo"], scale=ex["scale"], skeys=ex["skeys"], sids=ex["sids"],
                shifts=None if shifts is None else np.ascontiguousarray(shifts, np.int32).reshape(C_, D))


# ----------------------------------------------------------------------------
# full scan (Sec. I)
# ----------------------------------------------------------------------------
def check_fullscan(S, g, m_dict, m_cur, t, K, w=None):
    fp, fc = S.fullscan_query_batch(dev(g), dev(m_dict), dev(m_cur), dev(t), K=K, ch_weights=w)
    torch.cuda.synchronize()
    d = O.dict_extract(m_dict, K)
    op, oc = O.fullscan(g, m_cur, K, d, O.centres_to_lin(t, ext_of(g)), w)
    assert np.array_equal(fp.cpu().numpy(), op)
    assert cost_close(fc.cpu().numpy(), oc)
    return op


def test_fullscan_sines_front_targets(S):
    g, m = synth.sines2d(128)
    t = synth.front_targets(m, 9)
    assert len(O.dict_extract(m, 9)) == 13376  # spans 13 tiles of 1024 + a ragged tail
    check_fullscan(S, g, m, m, t, 9)


def test_fullscan_rgb_weighted_and_random_targets(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=2)
    t = np.concatenate([synth.front_targets(m, 7, cap=40, cfg=2), synth.random_targets(m, 7, 30, cfg=2)])
    check_fullscan(S, g, m, m, t, 7)
    check_fullscan(S, g, m, m, t, 7, w=np.array([1.0, 2.0, 0.5], np.float32))


def test_fullscan_exact_ties_lowest_id(S):
    rng = np.random.default_rng(5)
    g = rng.random((40, 40, 1)).astype(np.float32)
    g[30:35, 30:35] = g[3:8, 3:8]
    g[20:25, 2:7] = g[3:8, 3:8]
    m = np.ones((40, 40), np.uint8)
    t = np.array([[32, 32], [4, 22], [5, 5]], np.int32)
    op = check_fullscan(S, g, m, m, t, 5)
    d = O.dict_extract(m, 5)
    assert d[op[0]] == 5 * 40 + 5 and d[op[1]] == 5 * 40 + 5


def test_fullscan_constant_grid(S):
    g = np.full((30, 30, 2), 0.25, np.float32)
    m = np.ones((30, 30), np.uint8)
    m[10:14, 10:14] = 0
    t = np.array([[12, 9], [3, 3], [26, 26]], np.int32)
    op = check_fullscan(S, g, m, m, t, 3)
    assert list(op) == [0, 0, 0]


def test_fullscan_3d(S):
    g, m = synth.spheres3d(24, block=4, missing=0.1)
    t = synth.front_targets(m, 5, cap=40, cfg=3)
    check_fullscan(S, g, m, m, t, 5)


def test_fullscan_invalid_centre_and_empty_batch(S):
    g, m = synth.sines2d(64)
    t = np.array([[1, 1], [30, 30], [63, 10]], np.int32)
    fp, fc = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=9)
    fp = fp.cpu().numpy()
    fc = fc.cpu().numpy()
    assert fp[0] == -1 and np.isnan(fc[0]) and fp[2] == -1
    assert fp[1] >= 0
    assert S.sfc_status() == S.SFC_EDEVICE
    assert S.sfc_status() == 0  # cleared
    fp, fc = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(np.zeros((0, 2), np.int32)), K=9)
    assert fp.numel() == 0


# ----------------------------------------------------------------------------
# index build (Sec. II.A-C)
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def rgb_index(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)
    K, C_, D, bits = 7, 8, 6, 12
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=16, pca_sample=0,
                           keep_intermediates=1)
    ex = S.sfc_index_export(ix, proj=True)
    assert S.sfc_status() == 0  # the eigen-solve converged on every index
    return dict(g=g, m=m, K=K, C=C_, D=D, bits=bits, ix=ix, ex=ex)


def test_index_dictionary_and_subsets(rgb_index):
    r = rgb_index
    assert np.array_equal(r["ex"]["dict"], O.dict_extract(r["m"], r["K"]))
    assert np.array_equal(r["ex"]["subsets"], O.subsets(2, r["K"], 0.6, r["C"]))


def test_index_pca_basis_close_to_oracle(rgb_index):
    r = rgb_index
    ex = r["ex"]
    d = ex["dict"]
    for cv in range(r["C"]):
        B, mu, ev, cov = O.pca(r["g"], r["K"], d, ex["subsets"][cv], 0, r["D"])
        # eigenvalues: FP64 throughout, different summation/rotation order
        D = r["D"]
        assert np.allclose(ex["evals"][cv][:D], ev[:D], rtol=1e-9, atol=1e-12 * ev[0])
        assert np.all(np.abs(ex["mean"][cv] - mu) <= np.spacing(np.abs(mu)))
        # eigenvectors with an eigen-gap: same direction and canonical sign
        gaps = np.minimum(np.abs(np.diff(ev[: r["D"] + 1])), np.r_[np.inf, np.abs(np.diff(ev[: r["D"]]))])
        for k in range(r["D"]):
            if gaps[k] > 1e-6 * ev[0]:
                assert np.abs(ex["basis"][cv][:, k] - B[:, k]).max() < 2e-6


@pytest.mark.parametrize("shift", [0.5, 0.2])
def test_index_pca_with_negative_values(S, shift):
    # grid values shifted below zero (all of them around 0.5, some at 0.2): the
    # moments then take the general two-sum path, from the first chunk or from
    # a later one on, and the eigenpairs still match the oracle's
    g, m = synth.voronoi2d(80, cfg=2, seed_sub=5)
    g = (g - np.float32(shift)).astype(np.float32)
    K, C_, D = 7, 4, 6
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=12, window=16, pca_sample=0)
    ex = S.sfc_index_export(ix)
    ix.close()
    assert S.sfc_status() == 0
    for cv in range(C_):
        B, mu, ev, _ = O.pca(g, K, ex["dict"], ex["subsets"][cv], 0, D)
        assert np.allclose(ex["evals"][cv][:D], ev[:D], rtol=1e-9, atol=1e-12 * ev[0])
        assert np.all(np.abs(ex["mean"][cv] - mu) <= np.spacing(np.abs(mu)))


def test_index_keys_bit_exact_from_common_basis(rgb_index):
    r = rgb_index
    ex = r["ex"]
    oix = O.build_index(r["g"], r["m"], r["K"], r["C"], r["D"], r["bits"], basis=ex["basis"], mean=ex["mean"])
    assert np.array_equal(oix["proj"], ex["proj"])
    assert np.array_equal(oix["lo"], ex["lo"]) and np.array_equal(oix["scale"], ex["scale"])
    assert np.array_equal(oix["keys"], ex["keys"])
    assert np.array_equal(oix["skeys"], ex["skeys"]) and np.array_equal(oix["sids"], ex["sids"])


def test_index_shifted_curves_and_sampled_pca(S):
    g, m = synth.voronoi2d(80, cfg=2, seed_sub=4)
    K, C_, D, bits = 5, 6, 5, 10
    rng = np.random.default_rng(3)
    sh = rng.integers(0, 1 << bits, (C_, D)).astype(np.int32)
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=8, pca_sample=500,
                           shifts=sh, keep_intermediates=1)
    ex = S.sfc_index_export(ix, proj=True)
    d = ex["dict"]
    B, mu, ev, _ = O.pca(g, K, d, ex["subsets"][0], 500, D)
    assert np.allclose(ex["evals"][0][:D], ev[:D], rtol=1e-9, atol=1e-12 * ev[0])
    oix = O.build_index(g, m, K, C_, D, bits, shifts=sh, basis=ex["basis"], mean=ex["mean"])
    assert np.array_equal(oix["keys"], ex["keys"])
    assert np.array_equal(oix["skeys"], ex["skeys"]) and np.array_equal(oix["sids"], ex["sids"])
    t = synth.front_targets(m, K, cap=30, cfg=2)
    qk, pos, cand, nc = S.sfc_query_candidates(ix, dev(g), dev(m), dev(t))
    oq = oracle_ix(ex, g, K, C_, D, bits, sh)
    lin = O.centres_to_lin(t, ext_of(g))
    for i in range(len(t)):
        rr = O.query(oq, g, m, lin[i], 8)
        assert np.array_equal(qk[i].cpu().numpy().view(np.uint64), rr["qkeys"])
        assert np.array_equal(cand[i, : nc[i]].cpu().numpy(), rr["cand"])
    ix.close()


def test_index_3d_truncated_keys(S):
    g, m = synth.spheres3d(24, block=4, missing=0.1)
    K, C_, D, bits = 5, 8, 6, 21  # 126 key bits -> top 64
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=12, pca_sample=0,
                           keep_intermediates=1)
    ex = S.sfc_index_export(ix, proj=True)
    assert np.array_equal(ex["dict"], O.dict_extract(m, K))
    assert np.array_equal(ex["subsets"], O.subsets(3, K, 0.6, C_))
    oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
    assert np.array_equal(oix["proj"], ex["proj"])
    assert np.array_equal(oix["skeys"], ex["skeys"]) and np.array_equal(oix["sids"], ex["sids"])
    t = synth.front_targets(m, K, cap=25, cfg=3)
    p, c = S.sfc_query_batch(ix, dev(g), dev(m), dev(t))
    lin = O.centres_to_lin(t, ext_of(g))
    p = p.cpu().numpy()
    c = c.cpu().numpy()
    for i in range(len(t)):
        rr = O.query(oix, g, m, lin[i], 12)
        assert p[i] == rr["pick"] and cost_close(c[i], rr["cost"])
    ix.close()


# ----------------------------------------------------------------------------
# queries (Fig. 1(b)-(d))
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("select", [0, 1])
def test_query_candidates_and_picks(S, rgb_index, select):
    r = rgb_index
    g, m, K = r["g"], r["m"], r["K"]
    W = 16
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=r["C"], dims=r["D"], bits=r["bits"], window=W,
                           pca_sample=0, select=select)
    ex = S.sfc_index_export(ix)
    oq = oracle_ix(ex, g, K, r["C"], r["D"], r["bits"])
    t = np.concatenate([synth.front_targets(m, K, cap=60, cfg=2), synth.random_targets(m, K, 20, cfg=2)])
    # a partly filled state: current mask differs from the dictionary mask
    cur = m.copy()
    cur[40:50, 40:50] = 1
    for mask in (m, cur):
        qk, pos, cand, nc = S.sfc_query_candidates(ix, dev(g), dev(mask), dev(t))
        pk, cs = S.sfc_query_batch(ix, dev(g), dev(mask), dev(t))
        qk, pos, cand, nc = (x.cpu().numpy() for x in (qk, pos, cand, nc))
        pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
        lin = O.centres_to_lin(t, ext_of(g))
        for i in range(len(t)):
            rr = O.query(oq, g, mask, lin[i], W, select=select)
            assert np.array_equal(qk[i].view(np.uint64), rr["qkeys"])
            assert np.array_equal(pos[i], rr["pos"])
            assert nc[i] == len(rr["cand"]) and np.array_equal(cand[i, : nc[i]], rr["cand"])
            assert np.all(cand[i, nc[i]:] == -1)
            assert pk[i] == rr["pick"] and cost_close(cs[i], rr["cost"])
    ix.close()


def test_query_window_covering_dictionary_equals_fullscan(S):
    g, m = synth.voronoi2d(48, cfg=2, seed_sub=8)
    K = 5
    N = len(O.dict_extract(m, K))
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=2, dims=4, bits=8, window=N, pca_sample=0)
    t = synth.front_targets(m, K, cap=50, cfg=2)
    pk, cs = S.sfc_query_batch(ix, dev(g), dev(m), dev(t))
    fp, fc = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=K)
    assert torch.equal(pk, fp) and cost_close(cs.cpu().numpy(), fc.cpu().numpy())
    ix.close()


def test_query_exact_ties_and_constant_grid(S):
    # several exact duplicates in the window: the FP64 band pass must return the
    # lowest id; a constant grid ties every candidate at cost 0
    rng = np.random.default_rng(9)
    g = rng.random((40, 40, 1)).astype(np.float32)
    for (y, x) in [(30, 30), (20, 2), (2, 30)]:
        g[y:y + 5, x:x + 5] = g[3:8, 3:8]
    m = np.ones((40, 40), np.uint8)
    N = len(O.dict_extract(m, 5))
    ix = S.sfc_index_build(dev(g), dev(m), K=5, curves=2, dims=3, bits=8, window=N, pca_sample=0)
    assert S.sfc_status() == 0  # white noise has no eigen-gap; the 15-value subsets are solved by Jacobi
    t = np.array([[32, 32], [4, 22], [5, 5], [20, 20]], np.int32)
    pk, cs = S.sfc_query_batch(ix, dev(g), dev(m), dev(t))
    d = O.dict_extract(m, 5)
    pk = pk.cpu().numpy()
    # copies centred at (5,5), (32,32), (4,22), (32,4): the last has the lowest
    # raster rank (row 4), so it is the pick for all three duplicate targets
    assert all(d[pk[i]] == 4 * 40 + 32 for i in range(3))
    op, oc = O.fullscan(g, m, 5, d, O.centres_to_lin(t, ext_of(g)))
    assert np.array_equal(pk, op) and cost_close(cs.cpu().numpy(), oc)
    ix.close()
    gc = np.full((24, 24, 3), 0.5, np.float32)
    mc = np.ones((24, 24), np.uint8)
    ix = S.sfc_index_build(dev(gc), dev(mc), K=3, curves=4, dims=2, bits=4, window=16, pca_sample=0)
    pk, cs = S.sfc_query_batch(ix, dev(gc), dev(mc), dev(np.array([[10, 10], [1, 1]], np.int32)))
    ex = S.sfc_index_export(ix)
    oq = oracle_ix(ex, gc, 3, 4, 2, 4)
    for i, c in enumerate([(10, 10), (1, 1)]):
        rr = O.query(oq, gc, mc, c[1] * 24 + c[0], 16)
        assert pk[i].item() == rr["pick"] and cs[i].item() == 0.0
    ix.close()


def test_query_dictionary_patches_cost_zero(S, rgb_index):
    r = rgb_index
    ex = r["ex"]
    ext = ext_of(r["g"])
    js = np.array([0, 5, len(ex["dict"]) // 2, len(ex["dict"]) - 1])
    t = O.lin_to_centres(ex["dict"][js], ext, 2).astype(np.int32)
    pk, cs = S.sfc_query_batch(r["ix"], dev(r["g"]), dev(r["m"]), dev(t))
    assert torch.all(cs == 0) and torch.all(pk.cpu() <= torch.from_numpy(js))


# ----------------------------------------------------------------------------
# fill loop (Sec. I, Fig. 1(a))
# ----------------------------------------------------------------------------
def run_fill(S, g, m, **kw):
    gd, md = dev(g), dev(m)
    steps, log = S.inpaint_run(gd, md, **kw)
    return gd.cpu().numpy(), md.cpu().numpy(), log.cpu().numpy(), steps


def test_fill_sines_fullscan_bit_identical(S):
    g, m = synth.sines2d(128)
    og, om, olog, osteps = O.inpaint(g, m, 9, mode=0, prio=0)
    gg, gm, glog, gsteps = run_fill(S, g, m, mode=S.SFC_MODE_FULLSCAN, K=9, priority=0)
    assert gsteps == osteps and np.array_equal(glog, olog)
    assert np.array_equal(gg, og) and gm.all()


def test_fill_rgb_criminisi_fullscan_bit_identical(S):
    g, m = synth.voronoi2d(56, cfg=2, seed_sub=9)
    og, om, olog, osteps = O.inpaint(g, m, 5, mode=0, prio=1)
    gg, gm, glog, gsteps = run_fill(S, g, m, mode=S.SFC_MODE_FULLSCAN, K=5, priority=1)
    assert gsteps == osteps and np.array_equal(glog, olog)
    assert np.array_equal(gg, og)


def test_fill_rgb_sfc_bit_identical(S):
    g, m = synth.voronoi2d(64, cfg=2, seed_sub=10)
    K, C_, D, bits, W = 5, 8, 5, 10, 12
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0)
    ex = S.sfc_index_export(ix)
    ix.close()
    oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
    og, om, olog, osteps = O.inpaint(g, m, K, mode=1, prio=1, ix=oix, W=W)
    gg, gm, glog, gsteps = run_fill(S, g, m, mode=S.SFC_MODE_SFC, K=K, curves=C_, dims=D, bits=bits, window=W,
                                    basis=ex["basis"], mean=ex["mean"], priority=1)
    assert gsteps == osteps and np.array_equal(glog, olog)
    assert np.array_equal(gg, og)


def test_fill_3d_and_max_steps(S):
    g, m = synth.spheres3d(20, block=4, missing=0.05)
    og, om, olog, osteps = O.inpaint(g, m, 3, mode=0, prio=0, max_steps=40)
    gg, gm, glog, gsteps = run_fill(S, g, m, mode=S.SFC_MODE_FULLSCAN, K=3, priority=0, max_steps=40)
    assert gsteps == osteps == 40 and np.array_equal(glog, olog) and np.array_equal(gg, og)


# ----------------------------------------------------------------------------
# the full paper-scale 2-D workload (1024^2 RGB, K=11, C=8, D=8, b=16, W=64)
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def big(S):
    g, m = synth.voronoi2d(1024, cfg=2)
    t = synth.front_targets(m, 11, cap=65536, cfg=2)
    gd, md, td = dev(g), dev(m), dev(t)
    ix = S.sfc_index_build(gd, md, K=11, curves=8, dims=8, bits=16, window=64, pca_sample=16384,
                           keep_intermediates=1)
    ex = S.sfc_index_export(ix, proj=True)
    assert S.sfc_status() == 0
    return dict(g=g, m=m, t=t, gd=gd, md=md, td=td, ix=ix, ex=ex)


def test_big_index_sorted_permutation_and_sampled_keys(big):
    ex, g = big["ex"], big["g"]
    C_, N = ex["skeys"].shape
    assert N > 800_000
    for cv in range(C_):
        assert np.all(ex["skeys"][cv][1:] >= ex["skeys"][cv][:-1])
        assert np.array_equal(np.sort(ex["sids"][cv]), np.arange(N, dtype=np.uint32))
        assert np.array_equal(ex["keys"][cv][ex["sids"][cv]], ex["skeys"][cv])
    rng = np.random.default_rng(0)
    ones = np.ones(big["m"].shape, np.uint8)
    for j in rng.choice(N, 64, replace=False):
        for cv in (0, 3, 7):
            y = O.project_query(g, ones, 11, ex["dict"][j], ex["subsets"][cv], ex["basis"][cv], ex["mean"][cv], 8)
            assert np.array_equal(y, ex["proj"][cv][j])
            q = O.quantise(y[None], 16, ex["lo"][cv], ex["scale"][cv])
            assert O.keys(q, 16)[0] == ex["keys"][cv][j]


@pytest.fixture(scope="module")
def opool():
    from oracle import parallel as OP

    ex = OP.make_pool()
    yield ex, OP.default_workers()
    ex.shutdown()


@pytest.fixture(scope="module")
def big_oracle(big, opool):
    """The oracle's index of the full workload, built from the GPU's exported
    basis (checkpoint split: everything downstream of the basis must be
    bit-exact), its indices built in parallel worker processes."""
    from oracle import parallel as OP

    ex = big["ex"]
    return OP.build_index(opool[0], big["g"], big["m"], 11, 8, 8, 16, basis=ex["basis"], mean=ex["mean"])


def test_big_oracle_index_bit_exact(big, big_oracle):
    # every projection, quantiser, key and both sorted arrays of all 8 indices
    ex, oix = big["ex"], big_oracle
    assert np.array_equal(oix["dict"], ex["dict"])
    assert np.array_equal(oix["proj"], ex["proj"])
    assert np.array_equal(oix["lo"], ex["lo"]) and np.array_equal(oix["scale"], ex["scale"])
    assert np.array_equal(oix["keys"], ex["keys"])
    assert np.array_equal(oix["skeys"], ex["skeys"]) and np.array_equal(oix["sids"], ex["sids"])


def test_big_all_queries_match_oracle(S, big, big_oracle, opool):
    # all 3,597 front targets: candidate sets bit-exact, picks equal, costs
    # within 1e-5 of the exact cost, against the oracle's own sorted arrays
    from oracle import parallel as OP

    g, m, t = big["g"], big["m"], big["t"]
    assert len(t) == 3597  # every front target of the initial mask (the 65,536 cap is not reached)
    pk, cs = S.sfc_query_batch(big["ix"], big["gd"], big["md"], big["td"])
    pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
    _, _, cand, nc = S.sfc_query_candidates(big["ix"], big["gd"], big["md"], big["td"])
    cand, nc = cand.cpu().numpy(), nc.cpu().numpy()
    lin = O.centres_to_lin(t, ext_of(g))
    op, oc, ocand = OP.query_batch(opool[0], opool[1], big_oracle, g, m, lin, 64)
    assert np.array_equal(pk, op)
    assert cost_close(cs, oc)
    for i in range(len(t)):
        assert np.array_equal(cand[i, : nc[i]], ocand[i]), i


def test_big_fullscan_256_match_oracle(S, big, opool):
    # 256 seeded targets: the tensor-core full scan (a3) equals the FP32 scan
    # (a2) bit for bit, and both equal the oracle's brute-force picks
    from oracle import parallel as OP

    g, m, t = big["g"], big["m"], big["t"]
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(len(t), 256, replace=False))
    td = dev(t[sel])
    fp, fc = S.fullscan_query_batch(big["gd"], big["md"], big["md"], td, K=11)
    hp, hc = S.fullscan_query_batch(big["gd"], big["md"], big["md"], td, K=11, precision=S.SFC_FP16)
    assert torch.equal(fp, hp) and torch.equal(fc.view(torch.int32), hc.view(torch.int32))
    op, oc = OP.fullscan(opool[0], opool[1], g, m, 11, big["ex"]["dict"], O.centres_to_lin(t[sel], ext_of(g)))
    assert np.array_equal(fp.cpu().numpy(), op) and cost_close(fc.cpu().numpy(), oc)
