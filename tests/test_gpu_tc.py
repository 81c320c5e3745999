"""The full scan with the tensor-core pre-score (precision SFC_FP16) vs the
oracle and vs the FP32 scan, through the C-ABI (needs a GB300).

Bars: every pre-score within its bound E_q of the exact pre-score (checked on
differences, which cancel the per-query constant: |ds_hat - dcost| <= 2 E_q);
picks equal to the oracle's; the reported cost equal, bit for bit, to the FP32
scan's (both are the FP32 cost of the exact argmin) and within COST_RTOL of the
oracle's exact FP64 cost.
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


def patch_offsets(ext, ndim, K):
    r = K // 2
    X, Y = int(ext[0]), int(ext[1])
    if ndim == 2:
        dy, dx = np.mgrid[-r:r + 1, -r:r + 1]
        return (dy * X + dx).ravel()
    dz, dy, dx = np.mgrid[-r:r + 1, -r:r + 1, -r:r + 1]
    return (dz * X * Y + dy * X + dx).ravel()


def cost_matrix(g, m, K, dict_lin, t_lin, w=None):
    """Exact masked costs sum m w (t - p)^2 in float64 (Sec. I), all pairs."""
    ndim, ext, ch = O.geometry(g)
    off = patch_offsets(ext, ndim, K)
    v = g.reshape(-1, ch).astype(np.float64)
    mk = m.reshape(-1).astype(np.float64)
    wv = np.ones(ch) if w is None else np.asarray(w, np.float64)
    P = v[dict_lin[:, None] + off[None, :]]  # N x P x ch
    out = np.empty((len(t_lin), len(dict_lin)))
    for i, tl in enumerate(t_lin):
        T = v[tl + off]
        km = mk[tl + off][:, None] * wv[None, :]
        out[i] = (((P - T[None]) ** 2) * km[None]).sum(axis=(1, 2))
    return out


def check_tc(S, g, m, t, K, w=None):
    gd, md, td = dev(g), dev(m), dev(t)
    hp, hc = S.fullscan_query_batch(gd, md, md, td, K=K, ch_weights=w, precision=S.SFC_FP16)
    fp, fc = S.fullscan_query_batch(gd, md, md, td, K=K, ch_weights=w)
    torch.cuda.synchronize()
    hp, hc, fp, fc = hp.cpu().numpy(), hc.cpu().numpy(), fp.cpu().numpy(), fc.cpu().numpy()
    d = O.dict_extract(m, K)
    op, oc = O.fullscan(g, m, K, d, O.centres_to_lin(t, O.geometry(g)[1]), w)
    assert np.array_equal(hp, op)
    assert np.array_equal(hp, fp)
    assert np.array_equal(hc.view(np.uint32), fc.view(np.uint32))
    ok = op >= 0
    e = oc[ok]
    assert np.all(np.abs(hc[ok].astype(np.float64) - e) <= COST_RTOL * np.abs(e))
    assert np.all((hc[ok] == 0) == (e == 0))
    return op


def test_tc_prescores_within_bound(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=2)
    K = 7
    t = np.concatenate([synth.front_targets(m, K, cap=100, cfg=2), synth.random_targets(m, K, 30, cfg=2)])
    assert len(t) == 130  # two 128-row query tiles, the second ragged
    d = O.dict_extract(m, K)
    N = len(d)
    assert N % 256 != 0 and N > 4 * 256  # several dictionary tiles and a ragged tail
    sc, E = S.sfc_tc_prescores(dev(g), dev(m), dev(m), dev(t), K=K, N=N)
    sc = sc.cpu().numpy().astype(np.float64)
    E = E.cpu().numpy()
    lin = O.centres_to_lin(t, O.geometry(g)[1])
    c = cost_matrix(g, m, K, d, lin)
    # the numpy cost matrix is the oracle's cost (sampled pairs)
    rng = np.random.default_rng(0)
    for i, j in zip(rng.integers(0, len(t), 20), rng.integers(0, N, 20)):
        assert abs(c[i, j] - O.cost64(g, m, K, lin[i], d[j])) <= 1e-12 * max(1.0, c[i, j])
    j0 = np.argmin(c, axis=1)
    ds = sc - sc[np.arange(len(t)), j0][:, None]
    dc = c - c[np.arange(len(t)), j0][:, None]
    err = np.abs(ds - dc).max(axis=1)
    assert np.all(err <= 2 * E)
    # the bound is useful: far below the typical cost (targets with known pixels)
    med = np.median(c, axis=1)
    assert np.all(E[med > 0] < 0.01 * med[med > 0])


def test_tc_prescores_weighted_within_bound(S):
    g, m = synth.voronoi2d(64, cfg=2, seed_sub=4)
    K, w = 5, np.array([1.0, 2.0, 0.5], np.float32)
    t = synth.front_targets(m, K, cap=60, cfg=2)
    d = O.dict_extract(m, K)
    sc, E = S.sfc_tc_prescores(dev(g), dev(m), dev(m), dev(t), K=K, N=len(d), ch_weights=w)
    sc = sc.cpu().numpy().astype(np.float64)
    E = E.cpu().numpy()
    c = cost_matrix(g, m, K, d, O.centres_to_lin(t, O.geometry(g)[1]), w)
    ds = sc - sc[:, :1]
    dc = c - c[:, :1]
    assert np.all(np.abs(ds - dc).max(axis=1) <= 2 * E)


def test_tc_fullscan_rgb_front_and_random(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=2)
    t = np.concatenate([synth.front_targets(m, 7, cap=100, cfg=2), synth.random_targets(m, 7, 30, cfg=2)])
    check_tc(S, g, m, t, 7)


def test_tc_fullscan_rgb_weighted(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=5)
    t = synth.front_targets(m, 9, cap=140, cfg=2)
    check_tc(S, g, m, t, 9, w=np.array([1.0, 2.0, 0.5], np.float32))


def test_tc_fullscan_sines(S):
    g, m = synth.sines2d(128)
    t = synth.front_targets(m, 9)
    check_tc(S, g, m, t, 9)


def test_tc_fullscan_exact_ties_lowest_id(S):
    rng = np.random.default_rng(5)
    g = rng.random((40, 40, 1)).astype(np.float32)
    g[30:35, 30:35] = g[3:8, 3:8]
    g[20:25, 2:7] = g[3:8, 3:8]
    m = np.ones((40, 40), np.uint8)
    t = np.array([[32, 32], [4, 22], [5, 5]], np.int32)
    op = check_tc(S, g, m, t, 5)
    d = O.dict_extract(m, 5)
    assert d[op[0]] == 5 * 40 + 5 and d[op[1]] == 5 * 40 + 5


def test_tc_fullscan_constant_grid_every_tile(S):
    g = np.full((40, 40, 2), 0.25, np.float32)
    m = np.ones((40, 40), np.uint8)
    m[10:14, 10:14] = 0
    t = np.array([[12, 9], [3, 3], [36, 36]], np.int32)
    assert list(check_tc(S, g, m, t, 3)) == [0, 0, 0]


def test_tc_fullscan_3d(S):
    g, m = synth.spheres3d(24, block=4, missing=0.1)
    t = synth.front_targets(m, 5, cap=40, cfg=3)
    check_tc(S, g, m, t, 5)


def test_tc_fullscan_invalid_centre(S):
    g, m = synth.sines2d(64)
    t = np.array([[1, 1], [30, 30], [63, 10]], np.int32)
    S.sfc_status()
    hp, hc = S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=9, precision=S.SFC_FP16)
    hp, hc = hp.cpu().numpy(), hc.cpu().numpy()
    assert hp[0] == -1 and np.isnan(hc[0]) and hp[2] == -1 and hp[1] >= 0
    assert S.sfc_status() == S.SFC_EDEVICE
    assert S.sfc_status() == 0


def test_tc_range_rejected(S):
    g, m = synth.sines2d(64)
    t = np.array([[30, 30]], np.int32)
    with pytest.raises(RuntimeError, match="out of range"):
        S.fullscan_query_batch(dev(g * 1000.0), dev(m), dev(m), dev(t), K=9, precision=S.SFC_FP16)
    bad = g.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(RuntimeError, match="out of range"):
        S.fullscan_query_batch(dev(bad), dev(m), dev(m), dev(t), K=9, precision=S.SFC_FP16)
    with pytest.raises(RuntimeError, match="out of range"):
        S.fullscan_query_batch(dev(g), dev(m), dev(m), dev(t), K=9, precision=S.SFC_FP16,
                               ch_weights=np.array([40000.0], np.float32))
    # the FP32 path takes the same large values
    fp, _ = S.fullscan_query_batch(dev(g * 1000.0), dev(m), dev(m), dev(t), K=9)
    assert fp.cpu().numpy()[0] >= 0
    assert S.sfc_status() == 0


def test_tc_big_sampled(S):
    """1024^2 RGB, K = 11 (N = 901,592): 256 front targets, FP16 path equal to
    the FP32 scan; 6 of them against the oracle."""
    g, m = synth.voronoi2d(1024, cfg=2)
    t = synth.front_targets(m, 11, cap=65536, cfg=2)
    rng = np.random.default_rng(3)
    sel = np.sort(rng.choice(len(t), 256, replace=False))
    gd, md, td = dev(g), dev(m), dev(t[sel])
    hp, hc = S.fullscan_query_batch(gd, md, md, td, K=11, precision=S.SFC_FP16)
    fp, fc = S.fullscan_query_batch(gd, md, md, td, K=11)
    hp, hc, fp, fc = hp.cpu().numpy(), hc.cpu().numpy(), fp.cpu().numpy(), fc.cpu().numpy()
    assert np.array_equal(hp, fp) and np.array_equal(hc.view(np.uint32), fc.view(np.uint32))
    sub = np.r_[0, 255, rng.choice(np.arange(1, 255), 4, replace=False)]
    d = O.dict_extract(m, 11)
    op, oc = O.fullscan(g, m, 11, d, O.centres_to_lin(t[sel][sub], O.geometry(g)[1]))
    assert np.array_equal(hp[sub], op)
    assert np.all(np.abs(hc[sub] - oc) <= COST_RTOL * oc)
    assert S.sfc_status() == 0
