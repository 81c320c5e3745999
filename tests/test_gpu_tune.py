"""The parameter search over (C, D, W) through the C-ABI (needs a GB300).

Bars: the table lists every configuration in order; each configuration's
acceleration error equals the one recomputed here from its own index's
answers and the full scan's exact picks on the same sample (bit for bit: the
same FP32 costs); widening the window never raises the error (nested windows
of one index); the chosen row follows the selection rule; with k-NN lists the
list gives k.
"""
import numpy as np
import pytest
import torch

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


def ae_of(cost, exact):
    out = []
    for c, e in zip(cost.astype(np.float32), exact.astype(np.float32)):
        if c == e:
            out.append(0.0)
        elif not e > 0:
            out.append(1.0)
        else:
            out.append(np.sqrt(np.float64(c)) / np.sqrt(np.float64(e)) - 1.0)
    acc = 0.0
    for v in out:  # in order, as the library sums
        acc += float(v)
    return acc / len(out)


@pytest.mark.parametrize("knn", [0, 24])
def test_autotune_table_errors_and_choice(S, knn):
    g, m = synth.voronoi2d(192, cfg=4, seed_sub=3)
    K = 9
    t = synth.front_targets(m, K, cap=400, cfg=4)
    gd, md, td = dev(g), dev(m), dev(t)
    curves, dims, wins = (2, 8), (4, 8), ((8, 64) if knn == 0 else (4, 24))
    base = dict(K=K, bits=16, pca_sample=0, knn=knn)
    best, table, k = S.sfc_autotune(gd, md, td, curves=curves, dims=dims, windows=wins, sample=100, reps=2,
                                    ae_max=0.02, **base)
    assert table.shape == (8, 5)
    want = [(c, d, w) for c in curves for d in dims for w in wins]
    assert [tuple(int(v) for v in r[:3]) for r in table] == want
    assert np.all(table[:, 3] > 0) and np.all(table[:, 4] >= 0)
    # the sample: every ceil(Q / 100)-th query; its exact picks from the full scan
    Q = len(t)
    step = -(-Q // 100)
    rows = np.arange(0, Q, step)
    _, ec = S.fullscan_query_batch(gd, md, md, dev(t[rows]), K=K)
    ec = ec.cpu().numpy()
    for r, (c, d, w) in zip(table, want):
        prm = dict(base, curves=c, dims=d, **({"knn": w} if knn else {"window": w}))
        ix = S.sfc_index_build(gd, md, **prm)
        _, cs = S.sfc_query_batch(ix, gd, md, td)
        ix.close()
        assert r[4] == ae_of(cs.cpu().numpy()[rows], ec), (c, d, w)
    # nested windows (or longer lists) of one index never raise the error
    for i in range(0, 8, 2):
        assert table[i + 1, 4] <= table[i, 4]
    assert k == S.sfc_tune_select(table[:, 3], table[:, 4], 0.02)
    key = "knn" if knn else "window"
    assert (best["curves"], best["dims"], best[key]) == tuple(int(v) for v in table[k, :3])
    assert S.sfc_status() == 0


def test_autotune_query_objective_and_refusals(S):
    g, m = synth.voronoi2d(128, cfg=4, seed_sub=4)
    t = synth.front_targets(m, 7, cap=200, cfg=4)
    gd, md, td = dev(g), dev(m), dev(t)
    best, table, k = S.sfc_autotune(gd, md, td, curves=(4,), dims=(6,), windows=(16, 32), sample=50, reps=1,
                                    objective=S.SFC_TUNE_QUERY, ae_max=1e9, K=7, pca_sample=0)
    assert k == int(np.argmin(table[:, 3])) or table[k, 3] == table[:, 3].min()
    # a configuration the build refuses (D above the subset length) names itself
    with pytest.raises(RuntimeError, match="D 200"):
        S.sfc_autotune(gd, md, td, curves=(4,), dims=(200,), windows=(16,), sample=50, reps=1, K=7, pca_sample=0)
    assert S.sfc_status() == 0
