"""The full-size large 3-D configuration (512^3 grey volume with 5 %
salt-and-pepper outliers, 20 % missing 16^3 blocks, 9x9x9 patches (n = 729),
8 curves, 8 dimensions, 8 bits per axis -> 64-bit keys, window 256) through
the C-ABI, checked against the oracle on sampled outputs (needs a GB300).

The dictionary holds ~5e7 entries: the sorted keys and ids are checked whole
(order, permutation); keys and queries on samples the oracle computes one by
one; full-scan picks by the oracle's exact cost of the pick and a sampled
lower bound (no sampled entry costs less); the tensor-core full scan (its
dictionary operand in 8 GB chunks at this size) equals the FP32 one.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_06326_gb300 import synth

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-5
K, C_, D, BITS, W = 9, 8, 8, 8, 256


@pytest.fixture(scope="module")
def big5():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1712_06326_gb300 import sfc

    torch.cuda.set_device(0)
    g, m = synth.spheres3d(512, cfg=5, block=16, missing=0.20, salt=0.05)
    t = synth.front_targets(m, K, cap=131072, cfg=5)
    gd, md, td = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (g, m, t))
    sfc.sfc_status()
    ix = sfc.sfc_index_build(gd, md, K=K, curves=C_, dims=D, bits=BITS, window=W, pca_sample=65536)
    ex = sfc.sfc_index_export(ix)
    yield dict(S=sfc, g=g, m=m, t=t, gd=gd, md=md, td=td, ix=ix, ex=ex)
    ix.close()


def test_big5_dictionary_sorted_keys_and_sampled_keys(big5):
    ex, g, m = big5["ex"], big5["g"], big5["m"]
    N = len(ex["dict"])
    assert N > 3e7
    r = K // 2
    unk = np.pad((m == 0).astype(np.int32), ((1, 0), (1, 0), (1, 0))).cumsum(0).cumsum(1).cumsum(2)
    Z, Y, X = m.shape
    zs, ys, xs = np.arange(r, Z - r), np.arange(r, Y - r), np.arange(r, X - r)
    z0, z1, y0, y1, x0, x1 = zs - r, zs + r + 1, ys - r, ys + r + 1, xs - r, xs + r + 1
    box = (unk[np.ix_(z1, y1, x1)] - unk[np.ix_(z0, y1, x1)] - unk[np.ix_(z1, y0, x1)] - unk[np.ix_(z1, y1, x0)] +
           unk[np.ix_(z0, y0, x1)] + unk[np.ix_(z0, y1, x0)] + unk[np.ix_(z1, y0, x0)] - unk[np.ix_(z0, y0, x0)])
    assert N == int((box == 0).sum())
    del unk, box
    assert np.all(np.diff(ex["dict"]) > 0)
    rng = np.random.default_rng(0)
    ones = np.ones(m.shape, np.uint8)
    for cv in range(C_):
        sk, si = ex["skeys"][cv], ex["sids"][cv]
        assert np.all(sk[1:] >= sk[:-1])
        assert np.all(np.bincount(si, minlength=N) == 1)
        eq = sk[1:] == sk[:-1]
        assert np.all(si[1:][eq] > si[:-1][eq])
        for j in rng.choice(N, 8, replace=False):
            y = O.project_query(g, ones, K, ex["dict"][j], ex["subsets"][cv], ex["basis"][cv], ex["mean"][cv], D)
            q = O.quantise(y[None], BITS, ex["lo"][cv], ex["scale"][cv])
            key = np.uint64(O.keys(q, BITS)[0])
            # the entry sits in the run of its key (8 bits per axis: long runs of equal keys)
            lo, hi = int(np.searchsorted(sk, key, "left")), int(np.searchsorted(sk, key, "right"))
            assert hi > lo and np.any(si[lo:hi] == j)
    assert big5["S"].sfc_status() == 0


def test_big5_sampled_queries_match_oracle(big5):
    S, ex, g, m, t = big5["S"], big5["ex"], big5["g"], big5["m"], big5["t"]
    assert len(t) == 131072
    pk, cs = S.sfc_query_batch(big5["ix"], big5["gd"], big5["md"], big5["td"])
    pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
    assert np.all(pk >= 0)
    ndim, ext, ch = O.geometry(g)
    oq = dict(ndim=ndim, ext=ext, ch=ch, K=K, C=C_, D=D, bits=BITS, dict=ex["dict"], N=len(ex["dict"]),
              subset=np.ascontiguousarray(ex["subsets"]), m=ex["subsets"].shape[1], basis=ex["basis"],
              mean=ex["mean"], lo=ex["lo"], scale=ex["scale"], skeys=ex["skeys"], sids=ex["sids"], shifts=None)
    lin = O.centres_to_lin(t, ext)
    rng = np.random.default_rng(1)
    for i in np.r_[0, len(t) - 1, rng.choice(len(t), 14, replace=False)]:
        rr = O.query(oq, g, m, lin[i], W)
        assert pk[i] == rr["pick"]
        assert abs(float(cs[i]) - rr["cost"]) <= COST_RTOL * rr["cost"] and (cs[i] == 0) == (rr["cost"] == 0)
    assert S.sfc_status() == 0


def test_big5_fullscan_fp32_oracle_and_tensor_chunks(big5):
    S, g, m, t = big5["S"], big5["g"], big5["m"], big5["t"]
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(len(t), 64, replace=False))
    td = torch.from_numpy(np.ascontiguousarray(t[sel])).cuda()
    fp, fc = S.fullscan_query_batch(big5["gd"], big5["md"], big5["md"], td, K=K)
    hp, hc = S.fullscan_query_batch(big5["gd"], big5["md"], big5["md"], td, K=K, precision=S.SFC_FP16)
    fp, fc, hp, hc = fp.cpu().numpy(), fc.cpu().numpy(), hp.cpu().numpy(), hc.cpu().numpy()
    assert np.array_equal(hp, fp) and np.array_equal(hc.view(np.uint32), fc.view(np.uint32))
    # properties of the exact pick that the oracle checks at any size (a whole
    # oracle scan takes minutes here): its exact cost is the reported one, and
    # no entry of a 200,000-entry sample of the dictionary costs less
    d = big5["ex"]["dict"]
    lin = O.centres_to_lin(t[sel], O.geometry(g)[1])
    sample = np.sort(rng.choice(len(d), 200_000, replace=False))
    for i in (0, 17, 63):
        c = O.cost64(g, m, K, lin[i], d[fp[i]])
        assert abs(float(fc[i]) - c) <= COST_RTOL * c
        _, smin = O.fullscan(g, m, K, d[sample], lin[i:i + 1])
        assert smin[0] >= c
    assert S.sfc_status() == 0
