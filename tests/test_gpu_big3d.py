"""The full-size 3-D configuration (256^3 grey volume, 15 % missing 8^3 blocks,
7x7x7 patches, 8 curves, 12 dimensions, 21 bits per axis -> top-64-bit keys,
window 128) through the C-ABI, checked against the oracle on sampled outputs
(needs a GB300).

Bars as in test_gpu_parity: sorted keys non-decreasing, ids a permutation,
sampled keys bit-exact (oracle projection + quantiser + Morton from the GPU's
basis), sampled query picks equal and costs within 1e-5 of the oracle's (the
oracle searching the GPU's sorted arrays), sampled full-scan picks equal; the
tensor-core full scan equal to the FP32 one.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_06326_gb300 import synth

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-5
K, C_, D, BITS, W = 7, 8, 12, 21, 128


@pytest.fixture(scope="module")
def big3d():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1712_06326_gb300 import sfc

    torch.cuda.set_device(0)
    g, m = synth.spheres3d(256)
    t = synth.front_targets(m, K, cap=131072, cfg=3)
    gd, md, td = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (g, m, t))
    sfc.sfc_status()
    ix = sfc.sfc_index_build(gd, md, K=K, curves=C_, dims=D, bits=BITS, window=W, pca_sample=65536)
    ex = sfc.sfc_index_export(ix)
    return dict(S=sfc, g=g, m=m, t=t, gd=gd, md=md, td=td, ix=ix, ex=ex)


def oracle_ix(ex, grid):
    ndim, ext, ch = O.geometry(grid)
    return dict(ndim=ndim, ext=ext, ch=ch, K=K, C=C_, D=D, bits=BITS, dict=ex["dict"], N=len(ex["dict"]),
                subset=np.ascontiguousarray(ex["subsets"]), m=ex["subsets"].shape[1], basis=ex["basis"],
                mean=ex["mean"], lo=ex["lo"], scale=ex["scale"], skeys=ex["skeys"], sids=ex["sids"], shifts=None)


def test_big3d_index_sorted_and_sampled_keys(big3d):
    ex, g, m = big3d["ex"], big3d["g"], big3d["m"]
    N = len(ex["dict"])
    assert N > 4_000_000
    # the dictionary (Sec. I): every centre whose 7^3 box is inside and fully
    # known, in raster order -- the count from a summed-volume table, sampled
    # entries checked one by one
    r = K // 2
    unk = np.pad((m == 0).astype(np.int64), ((1, 0), (1, 0), (1, 0))).cumsum(0).cumsum(1).cumsum(2)
    Z, Y, X = m.shape
    zs, ys, xs = np.arange(r, Z - r), np.arange(r, Y - r), np.arange(r, X - r)
    z0, z1 = zs - r, zs + r + 1
    y0, y1 = ys - r, ys + r + 1
    x0, x1 = xs - r, xs + r + 1
    box = (unk[np.ix_(z1, y1, x1)] - unk[np.ix_(z0, y1, x1)] - unk[np.ix_(z1, y0, x1)] - unk[np.ix_(z1, y1, x0)] +
           unk[np.ix_(z0, y0, x1)] + unk[np.ix_(z0, y1, x0)] + unk[np.ix_(z1, y0, x0)] - unk[np.ix_(z0, y0, x0)])
    assert N == int((box == 0).sum())
    assert np.all(np.diff(ex["dict"]) > 0)
    for j in np.r_[0, N - 1, np.random.default_rng(7).choice(N, 200, replace=False)]:
        c = O.lin_to_centres(np.array([ex["dict"][j]]), O.geometry(g)[1], 3)[0]
        assert np.all(c >= r) and np.all(c < np.array([X, Y, Z]) - r)
        assert m[c[2] - r:c[2] + r + 1, c[1] - r:c[1] + r + 1, c[0] - r:c[0] + r + 1].all()
    rng = np.random.default_rng(0)
    ones = np.ones(m.shape, np.uint8)
    for cv in range(C_):
        sk, si = ex["skeys"][cv], ex["sids"][cv]
        assert np.all(sk[1:] >= sk[:-1])
        assert np.array_equal(np.sort(si), np.arange(N, dtype=np.uint32))
        # equal keys keep ascending ids (stable sort from id order)
        eq = sk[1:] == sk[:-1]
        assert np.all(si[1:][eq] > si[:-1][eq])
        inv = np.empty(N, np.int64)
        inv[si] = np.arange(N)
        for j in rng.choice(N, 16 if cv % 3 else 48, replace=False):
            y = O.project_query(g, ones, K, ex["dict"][j], ex["subsets"][cv], ex["basis"][cv], ex["mean"][cv], D)
            q = O.quantise(y[None], BITS, ex["lo"][cv], ex["scale"][cv])
            assert O.keys(q, BITS)[0] == sk[inv[j]]
    assert big3d["S"].sfc_status() == 0


def test_big3d_sampled_queries_match_oracle(big3d):
    S, ex, g, m, t = big3d["S"], big3d["ex"], big3d["g"], big3d["m"], big3d["t"]
    assert 10_000 < len(t) <= 131072
    pk, cs = S.sfc_query_batch(big3d["ix"], big3d["gd"], big3d["md"], big3d["td"])
    pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
    assert np.all(pk >= 0)
    oq = oracle_ix(ex, g)
    lin = O.centres_to_lin(t, O.geometry(g)[1])
    rng = np.random.default_rng(1)
    for i in np.r_[0, len(t) - 1, rng.choice(len(t), 30, replace=False)]:
        rr = O.query(oq, g, m, lin[i], W)
        assert pk[i] == rr["pick"]
        assert abs(float(cs[i]) - rr["cost"]) <= COST_RTOL * rr["cost"] and (cs[i] == 0) == (rr["cost"] == 0)
    assert S.sfc_status() == 0


def test_big3d_sampled_fullscan_fp32_and_tensor(big3d):
    S, g, m, t = big3d["S"], big3d["g"], big3d["m"], big3d["t"]
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(len(t), 256, replace=False))
    td = torch.from_numpy(np.ascontiguousarray(t[sel])).cuda()
    fp, fc = S.fullscan_query_batch(big3d["gd"], big3d["md"], big3d["md"], td, K=K)
    hp, hc = S.fullscan_query_batch(big3d["gd"], big3d["md"], big3d["md"], td, K=K, precision=S.SFC_FP16)
    fp, fc, hp, hc = fp.cpu().numpy(), fc.cpu().numpy(), hp.cpu().numpy(), hc.cpu().numpy()
    assert np.array_equal(hp, fp) and np.array_equal(hc.view(np.uint32), fc.view(np.uint32))
    sub = np.array([97])  # the oracle needs ~30 s per query at this size
    op, oc = O.fullscan(g, m, K, big3d["ex"]["dict"], O.centres_to_lin(t[sel][sub], O.geometry(g)[1]))
    assert np.array_equal(fp[sub], op)
    assert np.all(np.abs(fc[sub] - oc) <= COST_RTOL * oc)
    assert S.sfc_status() == 0
