"""Indices keyed by the Hilbert curve (curve = SFC_CURVE_HILBERT) vs the oracle,
through the C-ABI (needs a GB300).

Bars: unsorted and sorted keys and sorted ids bit-exact (the oracle rebuilt
from the GPU's exported basis), query keys, positions and candidate sets
bit-exact, picks equal, costs within 1e-5 of the oracle's exact cost.
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


def run_case(S, g, m, t, K, C_, D, bits, W, shifts=None, select=0):
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0,
                           curve=S.SFC_CURVE_HILBERT, shifts=shifts, select=select, keep_intermediates=1)
    ex = S.sfc_index_export(ix, proj=True)
    oix = O.build_index(g, m, K, C_, D, bits, shifts=shifts, basis=ex["basis"], mean=ex["mean"], curve=1)
    assert np.array_equal(oix["keys"], ex["keys"])
    assert np.array_equal(oix["skeys"], ex["skeys"]) and np.array_equal(oix["sids"], ex["sids"])
    # Hilbert keys differ from the z-curve keys of the same points
    mk = O.keys(oix["q"][0], bits, None if shifts is None else shifts[0])
    assert not np.array_equal(mk, ex["keys"][0])
    qk, pos, cand, ncand = S.sfc_query_candidates(ix, dev(g), dev(m), dev(t))
    pk, cs = S.sfc_query_batch(ix, dev(g), dev(m), dev(t))
    qk, pos = qk.cpu().numpy().view(np.uint64), pos.cpu().numpy()
    cand, ncand = cand.cpu().numpy(), ncand.cpu().numpy()
    pk, cs = pk.cpu().numpy(), cs.cpu().numpy()
    for i, tl in enumerate(O.centres_to_lin(t, O.geometry(g)[1])):
        r = O.query(oix, g, m, tl, W, select=select)
        assert np.array_equal(qk[i], r["qkeys"]) and np.array_equal(pos[i], r["pos"])
        assert np.array_equal(cand[i, :ncand[i]], r["cand"])
        assert pk[i] == r["pick"]
        assert abs(float(cs[i]) - r["cost"]) <= COST_RTOL * r["cost"] and (cs[i] == 0) == (r["cost"] == 0)
    assert S.sfc_status() == 0
    ix.close()


def test_hilbert_rgb(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)
    t = np.concatenate([synth.front_targets(m, 7, cap=50, cfg=2), synth.random_targets(m, 7, 14, cfg=2)])
    run_case(S, g, m, t, 7, 8, 6, 12, 16)


def test_hilbert_shifts_and_select_best(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=4)
    t = synth.front_targets(m, 7, cap=40, cfg=2)
    sh = np.random.default_rng(3).integers(0, 1 << 10, (8, 6)).astype(np.int32)
    run_case(S, g, m, t, 7, 8, 6, 10, 24, shifts=sh, select=1)


def test_hilbert_3d_truncated_and_exact_64(S):
    g, m = synth.spheres3d(32, block=4, missing=0.1)
    t = synth.front_targets(m, 5, cap=30, cfg=3)
    run_case(S, g, m, t, 5, 4, 12, 21, 32)  # 252 bits -> top 64
    run_case(S, g, m, t, 5, 4, 16, 4, 32)   # exactly 64 bits


def test_hilbert_with_knn_rejected(S):
    g, m = synth.sines2d(64)
    with pytest.raises(RuntimeError, match="z-curve"):
        S.sfc_index_build(dev(g), dev(m), K=9, curves=2, dims=4, bits=8, window=8, knn=8,
                          curve=S.SFC_CURVE_HILBERT)
