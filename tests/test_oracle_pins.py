"""Pins of the CPU oracle against facts the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: hand-worked
examples (tests/golden), closed forms, invariants the paper states, special
cases that reduce to an independent library routine (LAPACK, numpy sort /
searchsorted), or brute force on tiny inputs.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1712_06326_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _grid(rng, Y, X, ch=1):
    return rng.random((Y, X, ch)).astype(np.float32)


# ----------------------------------------------------------------------------
# dictionary (Sec. I: the fully known patches)
# ----------------------------------------------------------------------------
def test_dict_count_closed_form():
    for (Y, X, K) in [(12, 12, 3), (20, 17, 5), (9, 9, 9), (8, 8, 9)]:
        m = np.ones((Y, X), np.uint8)
        d = O.dict_extract(m, K)
        assert len(d) == max(0, X - K + 1) * max(0, Y - K + 1)
        assert np.all(np.diff(d) > 0)  # raster order


def test_dict_single_hole_removes_box():
    Y, X, K = 30, 40, 5
    m = np.ones((Y, X), np.uint8)
    m[12, 20] = 0
    d = O.dict_extract(m, K)
    assert len(d) == (X - K + 1) * (Y - K + 1) - K * K
    xs, ys = d % X, d // X
    assert not np.any((np.abs(xs - 20) <= 2) & (np.abs(ys - 12) <= 2))


def test_dict_3d_count():
    m = np.ones((7, 8, 9), np.uint8)
    d = O.dict_extract(m, 3)
    assert len(d) == 7 * 6 * 5
    m[3, 4, 4] = 0
    assert len(O.dict_extract(m, 3)) == 7 * 6 * 5 - 27


# ----------------------------------------------------------------------------
# masked L2 cost (Sec. II after Fig. 1) and full scan (Sec. I)
# ----------------------------------------------------------------------------
def test_cost_closed_form_constant_offset():
    # target - source = delta (dyadic, exact) at every known element:
    # cost = n_known * delta^2 exactly; unknown pixels contribute 0
    rng = np.random.default_rng(0)
    K = 5
    g = np.zeros((20, 20, 3), np.float32)
    base = (rng.integers(0, 64, (K, K, 3)) / 64.0).astype(np.float32)
    g[2:7, 2:7] = base
    g[10:15, 11:16] = base + np.float32(0.25)
    m = np.ones((20, 20), np.uint8)
    t = 12 * 20 + 13
    s = 4 * 20 + 4
    assert O.cost64(g, m, K, t, s) == pytest.approx(K * K * 3 * 0.0625, abs=0)
    m[10, 11] = 0
    m[14, 15] = 0
    assert O.cost64(g, m, K, t, s) == (K * K - 2) * 3 * 0.0625
    w = np.array([1.0, 2.0, 4.0], np.float32)
    assert O.cost64(g, m, K, t, s, w) == (K * K - 2) * 0.0625 * 7


def test_cost_ignores_unknown_target_values():
    rng = np.random.default_rng(1)
    g = _grid(rng, 16, 16)
    m = np.ones((16, 16), np.uint8)
    m[6:9, 6:9] = 0
    c1 = O.cost64(g, m, 5, 8 * 16 + 8, 3 * 16 + 12)
    g2 = g.copy()
    g2[6:9, 6:9] = 123.0
    assert O.cost64(g2, m, 5, 8 * 16 + 8, 3 * 16 + 12) == c1


def test_cost_brute_force_tiny_enumeration():
    # tiny grid, every pair: cost >= 0, cost(p, p) = 0 for fully known p,
    # symmetric for fully known pairs, and triangle-type bound sqrt-norm
    rng = np.random.default_rng(2)
    g = _grid(rng, 10, 10)
    m = np.ones((10, 10), np.uint8)
    d = O.dict_extract(m, 3)
    C = np.array([[O.cost64(g, m, 3, a, b) for b in d] for a in d])
    assert np.all(C >= 0)
    assert np.all(np.diag(C) == 0)
    assert np.array_equal(C, C.T)
    S = np.sqrt(C)
    for i in range(0, len(d), 7):
        assert np.all(S[i][:, None] <= S[i][None, :] + S + 1e-12)


# ----------------------------------------------------------------------------
# L1 cost (Sec. III.K)
# ----------------------------------------------------------------------------
def test_l1_cost_closed_form_constant_offset():
    # target - source = +-delta (dyadic) at every known element: L1 = n_known w delta
    rng = np.random.default_rng(30)
    K = 5
    g = np.zeros((20, 20, 3), np.float32)
    base = (rng.integers(0, 64, (K, K, 3)) / 64.0).astype(np.float32)
    sign = np.where(rng.random((K, K, 3)) < 0.5, -1.0, 1.0).astype(np.float32)
    g[2:7, 2:7] = base
    g[10:15, 11:16] = base + np.float32(0.25) * sign
    m = np.ones((20, 20), np.uint8)
    t, s_ = 12 * 20 + 13, 4 * 20 + 4
    assert O.cost64(g, m, K, t, s_, norm=1) == K * K * 3 * 0.25
    m[10, 11] = 0
    m[14, 15] = 0
    w = np.array([1.0, 2.0, 4.0], np.float32)
    assert O.cost64(g, m, K, t, s_, w, norm=1) == (K * K - 2) * 0.25 * 7
    assert O.cost64(g, m, K, t, s_, w) == (K * K - 2) * 0.0625 * 7  # L2 unchanged


def test_l1_fullscan_against_numpy_brute_force():
    rng = np.random.default_rng(31)
    g = rng.random((14, 15, 2)).astype(np.float32)
    m = np.ones((14, 15), np.uint8)
    m[5:8, 6:9] = 0
    K, r = 3, 1
    d = O.dict_extract(m, K)
    w = np.array([0.5, 3.0], np.float32)
    t = np.array([[6, 4], [9, 7], [2, 2], [13, 12]], np.int64)
    lin = O.centres_to_lin(t, O.geometry(g)[1])
    p, c = O.fullscan(g, m, K, d, lin, w, norm=1)
    X = g.shape[1]
    for i, tl in enumerate(lin):
        ty, tx = divmod(int(tl), X)
        T = g[ty - r:ty + r + 1, tx - r:tx + r + 1].astype(np.float64)
        km = m[ty - r:ty + r + 1, tx - r:tx + r + 1].astype(np.float64)[..., None]
        costs = []
        for j in d:
            sy, sx = divmod(int(j), X)
            P = g[sy - r:sy + r + 1, sx - r:sx + r + 1].astype(np.float64)
            costs.append(float((np.abs(T - P) * km * w.astype(np.float64)).sum()))
        costs = np.array(costs)
        assert p[i] == int(np.argmin(costs))  # first minimum = lowest id
        assert abs(c[i] - costs.min()) <= 1e-12 * max(1.0, costs.min())


def test_l1_is_a_metric_on_known_patches():
    rng = np.random.default_rng(32)
    g = _grid(rng, 10, 10)
    m = np.ones((10, 10), np.uint8)
    d = O.dict_extract(m, 3)
    C = np.array([[O.cost64(g, m, 3, a, b, norm=1) for b in d] for a in d])
    assert np.all(np.diag(C) == 0) and np.array_equal(C, C.T) and np.all(C >= 0)
    for i in range(0, len(d), 7):
        assert np.all(C[i][:, None] <= C[i][None, :] + C + 1e-12)


def test_l1_fill_one_pixel_hole_uses_bruteforce_pick():
    rng = np.random.default_rng(33)
    g = _grid(rng, 20, 20)
    m = np.ones((20, 20), np.uint8)
    m[9, 11] = 0
    d = O.dict_extract(m, 3)
    out, mo, log, steps = O.inpaint(g, m, 3, mode=0, norm=1)
    assert steps == 1 and mo.all()
    cx, cy, j = log[0]
    p, c = O.fullscan(g, m, 3, d, np.array([cy * 20 + cx]), norm=1)
    assert j == p[0]


def test_fullscan_exact_duplicate_tie_to_lowest_id():
    rng = np.random.default_rng(3)
    g = _grid(rng, 24, 24)
    # plant the patch around (5,5) again around (18,16): exact duplicates
    g[15:18, 17:20] = g[4:7, 4:7]
    m = np.ones((24, 24), np.uint8)
    d = O.dict_extract(m, 3)
    t = 16 * 24 + 18
    pick, cost = O.fullscan(g, m, 3, d, np.array([t]))
    assert cost[0] == 0.0
    assert d[pick[0]] == 5 * 24 + 5  # the lower-id duplicate, not the target itself


def test_fullscan_constant_grid_picks_zero():
    g = np.full((12, 12, 2), 0.375, np.float32)
    m = np.ones((12, 12), np.uint8)
    m[5:7, 5:7] = 0
    d = O.dict_extract(m, 3)
    pick, cost = O.fullscan(g, m, 3, d, np.array([6 * 12 + 6, 2 * 12 + 9]))
    assert list(pick) == [0, 0] and list(cost) == [0.0, 0.0]


def test_fullscan_planted_minimum():
    # every source differs from the target by >= 0.5 in one element except one
    rng = np.random.default_rng(4)
    K = 3
    g = (rng.integers(0, 4, (16, 16, 1)) / 4.0).astype(np.float32)
    m = np.ones((16, 16), np.uint8)
    d = O.dict_extract(m, K)
    t = 8 * 16 + 8
    costs = np.array([O.cost64(g, m, K, t, s) for s in d])
    costs[d == t] = np.inf
    pick, cost = O.fullscan(g, m, K, d, np.array([t]))
    # the full scan includes the target itself (cost 0) -> pick it
    assert d[pick[0]] == t and cost[0] == 0
    # with the target's own patch made unknown-centred the minimum is the brute one
    m2 = m.copy()
    m2[8, 8] = 0
    d2 = O.dict_extract(m, K)
    costs2 = np.array([O.cost64(g, m2, K, t, s) for s in d2])
    p2, c2 = O.fullscan(g, m2, K, d2, np.array([t]))
    assert c2[0] == costs2.min() and p2[0] == int(np.argmin(costs2))


# ----------------------------------------------------------------------------
# subsets (Fig. 2)
# ----------------------------------------------------------------------------
def _gold_subsets():
    rows = []
    for line in open(os.path.join(GOLD, "subsets_K3.txt")):
        if line.startswith("#") or not line.strip():
            continue
        _, pix = line.strip().split(";")
        rows.append([int(v) for v in pix.split(",")])
    return np.array(rows)


def test_subsets_hand_worked_K3():
    assert np.array_equal(O.subsets(2, 3, 0.5, 8), _gold_subsets())


def test_subsets_sizes_and_symmetry():
    for K, frac, m in [(9, 0.6, 49), (11, 0.6, 73), (7, 0.6, 29), (13, 0.6, 101)]:
        S = O.subsets(2, K, frac, 8)
        assert S.shape == (8, m)
        sets = [set(r) for r in S]
        # geometric symmetry of the anchors: the set sizes are equal and each
        # corner/edge subset maps onto its mirror under the patch's reflections
        # up to tie-breaking (equal distance shells differ by at most the last shell)
        for cv in range(8):
            pts = np.array([[p % K, p // K] for p in S[cv]])
            assert len(set(S[cv])) == m
            assert np.all(pts >= 0) and np.all(pts < K)
        # top-middle vs bottom-middle: mirror in y, same multiset of distances
        def d2(anchor, p):
            return (2 * (p % K) + 1 - anchor[0]) ** 2 + (2 * (p // K) + 1 - anchor[1]) ** 2
        top = sorted(d2((K, 0), p) for p in S[0])
        bot = sorted(d2((K, 2 * K), p) for p in S[2])
        assert top == bot
    # c = 1 covers the whole patch
    assert np.array_equal(O.subsets(2, 5, 1.0, 8)[3], np.arange(25))


def test_subsets_3d_corners():
    S = O.subsets(3, 3, 1.0 / 27.0, 14)
    # the single nearest voxel of each corner is that corner voxel
    corners = [0, 2, 6, 8, 18, 20, 24, 26]
    assert [int(r[0]) for r in S[:8]] == corners
    # face middles -> face-centre voxels z-, z+, y-, y+, x-, x+
    assert [int(r[0]) for r in S[8:]] == [4, 22, 10, 16, 12, 14]


# ----------------------------------------------------------------------------
# Jacobi eigen-solve and PCA (Sec. II.A)
# ----------------------------------------------------------------------------
def test_jacobi_2x2_closed_form():
    for a, b, d in [(2.0, 1.0, 3.0), (1.0, -0.5, 1.0), (5.0, 1e-3, -2.0), (0.0, 1.0, 0.0)]:
        ev, V, _ = O.jacobi(np.array([[a, b], [b, d]]))
        mid, rad = (a + d) / 2, np.hypot((a - d) / 2, b)
        assert sorted(ev) == pytest.approx([mid - rad, mid + rad], rel=1e-14, abs=1e-15)


def test_jacobi_diagonal_is_fixed_point():
    A = np.diag([3.0, -1.0, 7.5, 0.0])
    ev, V, sw = O.jacobi(A)
    assert list(ev) == [3.0, -1.0, 7.5, 0.0]
    assert np.array_equal(V, np.eye(4)) and sw == 0


@pytest.mark.parametrize("n", [3, 10, 57])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n + 5, n))
    A = X.T @ X / n
    ev, V, _ = O.jacobi(A)
    ref = np.linalg.eigvalsh(A)
    assert np.sort(ev) == pytest.approx(ref, rel=1e-11, abs=1e-12 * ref.max())
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12
    assert np.abs(A @ V - V * ev).max() < 1e-11 * ref.max()


def test_pca_covariance_and_basis():
    rng = np.random.default_rng(7)
    g = _grid(rng, 30, 30, 3)
    m = np.ones((30, 30), np.uint8)
    K, D = 5, 4
    d = O.dict_extract(m, K)
    sub = O.subsets(2, K, 0.6, 8)[5]
    B, mu, ev, cov = O.pca(g, K, d, sub, 0, D)
    # independent gather with numpy slicing + numpy covariance (LAPACK-free)
    xs, ys = d % 30, d // 30
    px, py = sub % K - K // 2, sub // K - K // 2
    X = np.stack([g[ys + py[i], xs + px[i], c] for i in range(len(sub)) for c in range(3)], 1).astype(np.float64)
    assert np.allclose(mu, X.mean(0).astype(np.float32), rtol=0, atol=1e-7)
    assert np.allclose(cov, np.cov(X, rowvar=False, bias=True), rtol=1e-12, atol=1e-15)
    ref = np.linalg.eigh(cov)
    assert ev[:D] == pytest.approx(ref[0][::-1][:D], rel=1e-11)
    for k in range(D):
        v = ref[1][:, ::-1][:, k]
        v = v * np.sign(v[np.argmax(np.abs(v))])
        assert np.abs(B[:, k] - v).max() < 1e-6
        assert B[np.argmax(np.abs(B[:, k])), k] > 0  # sign convention


def test_pca_sample_is_every_step_th_entry():
    rng = np.random.default_rng(8)
    g = _grid(rng, 20, 20)
    m = np.ones((20, 20), np.uint8)
    d = O.dict_extract(m, 3)
    sub = O.subsets(2, 3, 0.6, 1)[0]
    N = len(d)
    S = 50
    step = -(-N // S)
    B1, mu1, ev1, cov1 = O.pca(g, 3, d, sub, S, 2)
    B2, mu2, ev2, cov2 = O.pca(g, 3, d[::step], sub, 0, 2)
    assert np.array_equal(cov1, cov2) and np.array_equal(B1, B2)


def test_pca_rank_one_closed_form():
    # grid linear in x and y with dyadic values (exact in FP32): every subset
    # vector is v(centre) * (1, ..., 1) + const, so the covariance is
    # Var(v) * 1 1^T: one eigenvalue s * Var(v), eigenvector 1/sqrt(s), rest 0
    Y, X = 24, 24
    yy, xx = np.mgrid[0:Y, 0:X]
    g = ((xx + 2 * yy) / 64.0).astype(np.float32)[..., None]
    m = np.ones((Y, X), np.uint8)
    d = O.dict_extract(m, 5)
    sub = O.subsets(2, 5, 0.6, 1)[0]
    s = len(sub)
    B, mu, ev, cov = O.pca(g, 5, d, sub, 0, 3)
    v = ((d % X) + 2 * (d // X)) / 64.0
    assert ev[0] == pytest.approx(s * v.var(), rel=1e-13)
    assert abs(ev[1]) < 1e-13 * ev[0]
    assert np.allclose(B[:, 0], 1.0 / np.sqrt(s), rtol=0, atol=1e-7)


# ----------------------------------------------------------------------------
# projection (Sec. II.A), quantisation and Morton keys (Sec. II.C)
# ----------------------------------------------------------------------------
def test_projection_matches_float64_matmul():
    rng = np.random.default_rng(9)
    g = _grid(rng, 25, 25, 3)
    m = np.ones((25, 25), np.uint8)
    K, D = 5, 6
    d = O.dict_extract(m, K)
    sub = O.subsets(2, K, 0.6, 8)[2]
    B, mu, _, _ = O.pca(g, K, d, sub, 0, D)
    y = O.project(g, K, d, sub, B, mu, D)
    xs, ys = d % 25, d // 25
    px, py = sub % K - K // 2, sub // K - K // 2
    Xm = np.stack([g[ys + py[i], xs + px[i], c] for i in range(len(sub)) for c in range(3)], 1).astype(np.float64)
    ref = (Xm - mu.astype(np.float64)) @ B.astype(np.float64)
    assert np.abs(y - ref).max() < 1e-5


def test_projection_selector_basis_is_exact_and_query_skips_unknown():
    rng = np.random.default_rng(10)
    g = _grid(rng, 12, 12)
    m = np.ones((12, 12), np.uint8)
    K = 3
    sub = np.arange(9, dtype=np.int32)
    B = np.zeros((9, 2), np.float32)
    B[4, 0] = 1.0  # centre pixel
    B[0, 1] = 1.0  # top-left pixel
    mu = np.full(9, 0.5, np.float32)
    y = O.project_query(g, m, K, 5 * 12 + 5, sub, B, mu, 2)
    assert y[0] == np.float32(g[5, 5, 0] - np.float32(0.5))
    assert y[1] == np.float32(g[4, 4, 0] - np.float32(0.5))
    m[4, 4] = 0
    y = O.project_query(g, m, K, 5 * 12 + 5, sub, B, mu, 2)
    assert y[1] == 0.0 and y[0] == np.float32(g[5, 5, 0] - np.float32(0.5))


def test_projection_is_a_fused_multiply_add_chain_in_subset_order():
    # Reading r7 of the projection arithmetic (Sec. II.A leaves it open): the
    # accumulator is updated by one fused multiply-add per subset value, in
    # subset order.  Values chosen so that the three plausible readings differ:
    # B0 = -1, x0 = 1 + 2^-11 gives acc = -(1 + 2^-11) exactly; then
    # B1 = x1 = 1 + 2^-12, whose exact product 1 + 2^-11 + 2^-24 is not a float.
    #   fused:            acc + B1 x1 rounded once          = 2^-24
    #   separate rounding: fl(B1 x1) = 1 + 2^-11 (tie to even) -> 0
    #   reversed order:   fl(B1 x1) first, then -(1 + 2^-11) -> 0
    a = np.float32(1 + 2.0 ** -11)
    b = np.float32(1 + 2.0 ** -12)
    assert np.float32(b * b) == a  # the product alone rounds to 1 + 2^-11
    g = np.full((5, 5, 1), 0.5, np.float32)
    g[1, 1, 0] = a  # patch pixel 0 of the centre (2, 2)
    g[1, 2, 0] = b  # patch pixel 1
    m = np.ones((5, 5), np.uint8)
    sub = np.arange(9, dtype=np.int32)
    B = np.zeros((9, 1), np.float32)
    B[0, 0] = -1.0
    B[1, 0] = b
    mu = np.zeros(9, np.float32)
    want = np.float32(2.0 ** -24)
    assert O.project_query(g, m, 3, 2 * 5 + 2, sub, B, mu, 1)[0] == want
    assert O.project(g, 3, np.array([2 * 5 + 2]), sub, B, mu, 1)[0, 0] == want


def test_quantise_closed_forms():
    y = np.array([[0.0], [1.0], [0.5], [0.25], [-3.0], [9.0]], np.float32)
    lo, sc = O.quant_params(y[:2], 8)
    assert lo[0] == 0.0 and sc[0] == 256.0
    q = O.quantise(y, 8, lo, sc)[:, 0]
    assert list(q) == [0, 255, 128, 64, 0, 255]
    lo, sc = O.quant_params(np.zeros((3, 2), np.float32), 4)
    assert list(sc) == [0.0, 0.0]
    assert np.all(O.quantise(np.ones((2, 2), np.float32), 4, lo, sc) == 0)


def test_morton_hand_worked_examples():
    n = 0
    for line in open(os.path.join(GOLD, "morton_examples.txt")):
        if line.startswith("#") or not line.strip():
            continue
        b, coords, key = line.strip().split(";")
        q = np.array([int(v) for v in coords.split(",")], np.uint32)
        assert O.morton(q, int(b)) == int(key), line
        n += 1
    assert n >= 8


def test_morton_shift_adds_a_bit():
    assert O.key_bits(3, 8, np.array([0, 0, 0])) == 8
    assert O.key_bits(3, 8, np.array([0, 5, 0])) == 9
    q = np.array([[1, 2]], np.uint32)
    k = O.keys(q, 2, np.array([1, 1]))
    assert int(k[0]) == O.morton(np.array([2, 3], np.uint32), 3)


def test_zorder_comparison_orders_like_morton_keys():
    # Sec. II.C: deciding by the axis with the highest differing bit gives the
    # same order as comparing full z-addresses
    rng = np.random.default_rng(11)
    for D in [1, 2, 3, 5, 8]:
        q = rng.integers(0, 256, (300, D)).astype(np.uint32)
        q[50:60] = q[0]  # equal points
        k = O.keys(q, 8)
        for _ in range(3000):
            a, b = rng.integers(0, 300, 2)
            assert O.zless(q[a], q[b]) == (int(k[a]) < int(k[b]))


def test_morton_box_interval_property():
    # Sec. II.D: every point of an axis-aligned box lies in the z-interval
    # [z(min), z(max)] -- the property the litmax/bigmin split relies on
    rng = np.random.default_rng(12)
    for _ in range(50):
        lo = rng.integers(0, 12, 2)
        hi = lo + rng.integers(0, 5, 2)
        zmin = O.morton(lo.astype(np.uint32), 4)
        zmax = O.morton(hi.astype(np.uint32), 4)
        for x in range(lo[0], hi[0] + 1):
            for y in range(lo[1], hi[1] + 1):
                assert zmin <= O.morton(np.array([x, y], np.uint32), 4) <= zmax


def test_sort_and_lower_bound_against_numpy():
    rng = np.random.default_rng(13)
    k = rng.integers(0, 50, 5000).astype(np.uint64)
    k[::7] = np.uint64(2 ** 63 + 5)
    sk, si = O.sort(k)
    ref = np.argsort(k, kind="stable")
    assert np.array_equal(si, ref) and np.array_equal(sk, k[ref])
    assert np.array_equal(np.sort(si), np.arange(len(k)))
    for key in [0, 1, 17, 49, 50, 2 ** 63 + 5, 2 ** 64 - 1]:
        assert O.lower_bound(sk, key) == int(np.searchsorted(sk, np.uint64(key), side="left"))


def test_knn_bruteforce_against_numpy():
    rng = np.random.default_rng(14)
    q = rng.integers(0, 16, (400, 3)).astype(np.uint32)
    query = np.array([7, 8, 9], np.uint32)
    ids, dist = O.knn_bruteforce(q, query, 20)
    d = ((q.astype(np.int64) - query.astype(np.int64)) ** 2).sum(1)
    ref = np.lexsort((np.arange(400), d))[:20]
    assert np.array_equal(ids, ref) and np.array_equal(dist, d[ref])


# ----------------------------------------------------------------------------
# SFC query (Fig. 1(b)-(d))
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_rgb():
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=3)
    ix = O.build_index(g, m, 7, 8, 6, 12, sample=0)
    return g, m, ix


def test_index_keys_sorted_and_permutation(small_rgb):
    g, m, ix = small_rgb
    for cv in range(ix["C"]):
        assert np.all(np.diff(ix["skeys"][cv].astype(object)) >= 0)
        assert np.array_equal(np.sort(ix["sids"][cv]), np.arange(ix["N"]))
        assert np.array_equal(ix["keys"][cv][ix["sids"][cv]], ix["skeys"][cv])
        eq = ix["skeys"][cv][1:] == ix["skeys"][cv][:-1]
        assert np.all(ix["sids"][cv][1:][eq] > ix["sids"][cv][:-1][eq])


def test_query_window_covering_dictionary_equals_fullscan(small_rgb):
    g, m, ix = small_rgb
    t = synth.front_targets(m, 7, cap=12, cfg=2)
    lin = O.centres_to_lin(t, ix["ext"])
    fp, fc = O.fullscan(g, m, 7, ix["dict"], lin)
    for i, tl in enumerate(lin):
        r = O.query(ix, g, m, tl, W=ix["N"])
        assert r["pick"] == fp[i] and r["cost"] == fc[i]
        assert np.array_equal(r["cand"], np.arange(ix["N"]))


def test_query_dictionary_patch_finds_itself(small_rgb):
    g, m, ix = small_rgb
    for j in [0, 17, ix["N"] // 2, ix["N"] - 1]:
        r = O.query(ix, g, m, ix["dict"][j], W=16)
        assert r["cost"] == 0.0
        assert r["pick"] <= j
        assert ix["dict"][r["pick"]] == ix["dict"][j] or O.cost64(g, m, 7, ix["dict"][j], ix["dict"][r["pick"]]) == 0


def test_query_candidate_set_structure(small_rgb):
    g, m, ix = small_rgb
    t = synth.front_targets(m, 7, cap=20, cfg=2)
    lin = O.centres_to_lin(t, ix["ext"])
    W = 10
    for tl in lin:
        r = O.query(ix, g, m, tl, W=W)
        c = r["cand"]
        assert len(c) <= ix["C"] * W and np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < ix["N"]
        want = set()
        for cv in range(ix["C"]):
            p = O.lower_bound(ix["skeys"][cv], r["qkeys"][cv])
            assert p == r["pos"][cv]
            s0 = min(max(p - W // 2, 0), ix["N"] - W)
            want |= set(ix["sids"][cv][s0:s0 + W].tolist())
        assert set(c.tolist()) == want
        costs = [O.cost64(g, m, 7, tl, ix["dict"][j]) for j in c]
        assert r["cost"] == min(costs) and r["pick"] == c[int(np.argmin(costs))]


# ----------------------------------------------------------------------------
# Hilbert keys (Skilling's transpose method): pinned by the curve's defining
# properties, not by a second implementation
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("D,b", [(2, 1), (2, 3), (3, 2), (4, 2), (2, 5), (5, 2), (3, 3)])
def test_hilbert_is_a_unit_step_bijection(D, b):
    side = 1 << b
    cells = np.stack(np.meshgrid(*[np.arange(side)] * D, indexing="ij"), -1).reshape(-1, D).astype(np.uint32)
    k = np.array([O.hilbert(c, b) for c in cells], dtype=np.uint64)
    assert len(np.unique(k)) == len(cells) and int(k.max()) == len(cells) - 1
    assert O.hilbert(np.zeros(D, np.uint32), b) == 0
    order = cells[np.argsort(k)].astype(np.int64)
    step = np.abs(np.diff(order, axis=0))
    # consecutive positions on the curve are neighbouring cells: one coordinate moves by one
    assert np.all(step.sum(1) == 1) and np.all(step.max(1) == 1)


def test_hilbert_nesting_and_top64_truncation():
    rng = np.random.default_rng(21)
    for _ in range(200):
        x = rng.integers(0, 1 << 17, 4).astype(np.uint32)
        # the cell of x one level up is visited as one block: H_17(x) / 2^4 = H_16(x >> 1);
        # D * b = 68 > 64, so the key of x is exactly that quotient
        assert O.hilbert(x, 17) == O.hilbert(x >> 1, 16)
        y = rng.integers(0, 1 << 8, 6).astype(np.uint32)
        assert O.hilbert(y, 8) >> 6 == O.hilbert(y >> 1, 7)
    # keys() with curve 1 applies the shifts and b + 1 bits like the Morton keys
    q = rng.integers(0, 1 << 8, (50, 3)).astype(np.uint32)
    sh = np.array([3, 0, 200], np.int32)
    want = [O.hilbert(r + sh.astype(np.uint32), 9) for r in q]
    assert np.array_equal(O.keys(q, 8, sh, curve=1), np.array(want, np.uint64))


def test_hilbert_query_window_covering_dictionary_equals_fullscan():
    g, m = synth.voronoi2d(64, cfg=2, seed_sub=9)
    ix = O.build_index(g, m, 7, 4, 6, 10, sample=0, curve=1)
    for cv in range(4):
        assert np.all(np.diff(ix["skeys"][cv].astype(object)) >= 0)
    t = synth.front_targets(m, 7, cap=10, cfg=2)
    lin = O.centres_to_lin(t, ix["ext"])
    fp, fc = O.fullscan(g, m, 7, ix["dict"], lin)
    for i, tl in enumerate(lin):
        r = O.query(ix, g, m, tl, W=ix["N"])
        assert r["pick"] == fp[i] and r["cost"] == fc[i]


# ----------------------------------------------------------------------------
# queries against an index built on another grid (a stored dictionary)
# ----------------------------------------------------------------------------
def test_cost64_2_same_grid_and_numpy():
    rng = np.random.default_rng(40)
    a = rng.random((20, 24, 3)).astype(np.float32)
    b = rng.random((17, 30, 3)).astype(np.float32)
    mb = (rng.random((17, 30)) < 0.8).astype(np.uint8)
    ma = np.ones((20, 24), np.uint8)
    K, r = 5, 2
    w = np.array([1.0, 0.5, 2.0], np.float32)
    for t, sidx in [(3 * 24 + 4, 10 * 24 + 12), (17 * 24 + 21, 2 * 24 + 2)]:
        assert O.cost64_2(a, ma, a, K, t, sidx, w) == O.cost64(a, ma, K, t, sidx, w)
    for (ty, tx), (sy, sx) in [((5, 9), (4, 7)), ((14, 27), (17, 21)), ((2, 2), (2, 2))]:
        T = b[ty - r:ty + r + 1, tx - r:tx + r + 1].astype(np.float64)
        km = mb[ty - r:ty + r + 1, tx - r:tx + r + 1].astype(np.float64)[..., None]
        Pp = a[sy - r:sy + r + 1, sx - r:sx + r + 1].astype(np.float64)
        for norm in (0, 1):
            d = T - Pp
            ref = float(((np.abs(d) if norm else d * d) * km * w).sum())
            got = O.cost64_2(b, mb, a, K, ty * 30 + tx, sy * 24 + sx, w, norm)
            assert abs(got - ref) <= 1e-12 * max(1.0, ref)


def test_query_dict_same_grid_equals_query(small_rgb):
    g, m, ix = small_rgb
    t = synth.front_targets(m, 7, cap=10, cfg=2)
    for tl in O.centres_to_lin(t, ix["ext"]):
        r1 = O.query(ix, g, m, tl, W=12)
        r2 = O.query_dict(ix, g, g, m, tl, 12)
        assert r1["pick"] == r2["pick"] and r1["cost"] == r2["cost"] and np.array_equal(r1["cand"], r2["cand"])


def test_query_dict_other_grid_full_window_is_bruteforce(small_rgb):
    g, m, ix = small_rgb
    g2, m2 = synth.voronoi2d(80, cfg=2, seed_sub=11)  # another image, another size
    t = synth.front_targets(m2, 7, cap=6, cfg=2)
    lin = O.centres_to_lin(t, O.geometry(g2)[1])
    for tl in lin:
        r = O.query_dict(ix, g, g2, m2, tl, ix["N"])
        costs = np.array([O.cost64_2(g2, m2, g, 7, tl, j) for j in ix["dict"]])
        assert r["pick"] == int(np.argmin(costs)) and r["cost"] == costs.min()


# ----------------------------------------------------------------------------
# SFC query with exact k-NN lists (Sec. II.D)
# ----------------------------------------------------------------------------
def _numpy_knn(qc, query, k):
    d = ((qc.astype(np.int64) - query.astype(np.int64)) ** 2).sum(1)
    return np.lexsort((np.arange(len(d)), d))[:k]


def test_query_knn_covering_dictionary_equals_fullscan(small_rgb):
    g, m, ix = small_rgb
    t = synth.front_targets(m, 7, cap=8, cfg=2)
    lin = O.centres_to_lin(t, ix["ext"])
    fp, fc = O.fullscan(g, m, 7, ix["dict"], lin)
    for i, tl in enumerate(lin):
        r = O.query_knn(ix, g, m, tl, k=ix["N"] + 5)
        assert r["pick"] == fp[i] and r["cost"] == fc[i]
        assert np.array_equal(r["cand"], np.arange(ix["N"]))


def test_query_knn_candidates_are_the_union_of_nearest_lists(small_rgb):
    g, m, ix = small_rgb
    t = np.concatenate([synth.front_targets(m, 7, cap=10, cfg=2), synth.random_targets(m, 7, 6, cfg=2)])
    lin = O.centres_to_lin(t, ix["ext"])
    k = 24
    for tl in lin:
        r = O.query_knn(ix, g, m, tl, k=k)
        want = set()
        for cv in range(ix["C"]):
            y = O.project_query(g, m, 7, tl, ix["subset"][cv], ix["basis"][cv], ix["mean"][cv], ix["D"])
            qq = O.quantise(y[None], ix["bits"], ix["lo"][cv], ix["scale"][cv])[0]
            want |= set(_numpy_knn(ix["q"][cv], qq, k).tolist())
        assert set(r["cand"].tolist()) == want and np.all(np.diff(r["cand"]) > 0)
        costs = [O.cost64(g, m, 7, tl, ix["dict"][j]) for j in r["cand"]]
        assert r["cost"] == min(costs) and r["pick"] == r["cand"][int(np.argmin(costs))]


def test_query_knn_dictionary_patch_finds_itself(small_rgb):
    g, m, ix = small_rgb
    for j in [0, 17, ix["N"] // 2, ix["N"] - 1]:
        r = O.query_knn(ix, g, m, ix["dict"][j], k=4)
        assert j in set(r["cand"].tolist()) or r["cost"] == 0.0
        assert r["cost"] == 0.0 and r["pick"] <= j


def test_query_knn_select_best_single_list(small_rgb):
    g, m, ix = small_rgb
    t = synth.front_targets(m, 7, cap=6, cfg=2)
    for tl in O.centres_to_lin(t, ix["ext"]):
        r = O.query_knn(ix, g, m, tl, k=9, select=1)
        assert 1 <= len(r["cand"]) <= 9


def test_query_select_best_uses_max_coverage(small_rgb):
    g, m, ix = small_rgb
    t = synth.front_targets(m, 7, cap=10, cfg=2)
    lin = O.centres_to_lin(t, ix["ext"])
    ext = ix["ext"]
    for tl in lin:
        r = O.query(ix, g, m, tl, W=8, select=1)
        x, y = tl % ext[0], tl // ext[0]
        cov = []
        for cv in range(ix["C"]):
            sub = ix["subset"][cv]
            cov.append(int(sum(m[y + p // 7 - 3, x + p % 7 - 3] for p in sub)))
        best = int(np.argmax(cov))
        assert r["pos"][best] >= 0 and sum(p >= 0 for p in r["pos"]) == 1


# ----------------------------------------------------------------------------
# fill loop (Sec. I; Fig. 1(a))
# ----------------------------------------------------------------------------
def test_fill_one_pixel_hole_uses_bruteforce_pick():
    rng = np.random.default_rng(15)
    g = _grid(rng, 20, 20)
    m = np.ones((20, 20), np.uint8)
    m[9, 11] = 0
    d = O.dict_extract(m, 3)
    out, mo, log, steps = O.inpaint(g, m, 3, mode=0)
    assert steps == 1 and mo.all()
    cx, cy, j = log[0]
    # first target (confidence priority): the lowest-index centre among the
    # front pixels with the most known pixels in their patch
    assert (cx, cy) == (11, 8)
    p, c = O.fullscan(g, m, 3, d, np.array([cy * 20 + cx]))
    assert j == p[0]
    s = d[j]
    assert out[9, 11, 0] == g[s // 20 + 1, s % 20, 0]


def test_fill_confidence_first_target_is_hole_corner_closed_form():
    g, m = synth.sines2d(48, hole=(20, 28))
    out, mo, log, steps = O.inpaint(g, m, 5, mode=0, max_steps=1)
    # front pixels next to a corner of the square hole overlap it least; the
    # lowest linear index among them is (x0, y0 - 1)
    assert tuple(log[0][:2]) == (20, 19)


def test_fill_runs_to_completion_and_replays():
    g, m = synth.sines2d(48, hole=(20, 28))
    out, mo, log, steps = O.inpaint(g, m, 5, mode=0)
    assert mo.all() and 1 <= steps <= 64
    # replaying the logged (centre, source) copies onto the input reproduces it
    d = O.dict_extract(m, 5)
    rg, rm = g.copy(), m.copy()
    for cx, cy, j in log:
        sy, sx = divmod(int(d[j]), 48)
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                if not rm[cy + dy, cx + dx]:
                    rg[cy + dy, cx + dx] = g[sy + dy, sx + dx]
                    rm[cy + dy, cx + dx] = 1
    assert np.array_equal(rg, out) and rm.all()
    # every filled value is a value of the original known image
    known_vals = set(g[m.astype(bool)].ravel().tolist())
    assert set(out[m == 0].ravel().tolist()) <= known_vals


def test_fill_sfc_mode_with_full_windows_equals_fullscan_mode():
    g, m = synth.voronoi2d(40, cfg=2, seed_sub=5)
    ix = O.build_index(g, m, 5, 4, 4, 8, sample=0)
    a = O.inpaint(g, m, 5, mode=0, max_steps=25)
    b = O.inpaint(g, m, 5, mode=1, ix=ix, W=ix["N"], max_steps=25)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[0], b[0])


def test_fill_knn_lists_covering_dictionary_equal_fullscan_mode():
    g, m = synth.voronoi2d(40, cfg=2, seed_sub=5)
    ix = O.build_index(g, m, 5, 4, 4, 8, sample=0)
    a = O.inpaint(g, m, 5, mode=0, max_steps=25)
    b = O.inpaint(g, m, 5, mode=1, ix=ix, knn=ix["N"], max_steps=25)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[0], b[0])


def test_fill_knn_first_step_picks_from_the_nearest_lists():
    # one step of the fill with k-NN lists (Sec. II.D): the pick is the exact
    # argmin over the union of every curve's k nearest entries in quantised space
    g, m = synth.voronoi2d(48, cfg=2, seed_sub=8)
    K, k = 5, 7
    ix = O.build_index(g, m, K, 4, 4, 8, sample=0)
    _, _, log, steps = O.inpaint(g, m, K, mode=1, ix=ix, knn=k, max_steps=1)
    assert steps == 1
    tl = int(O.centres_to_lin(log[:1, :2], ix["ext"])[0])
    want = set()
    for cv in range(ix["C"]):
        y = O.project_query(g, m, K, tl, ix["subset"][cv], ix["basis"][cv], ix["mean"][cv], ix["D"])
        qq = O.quantise(y[None], ix["bits"], ix["lo"][cv], ix["scale"][cv])[0]
        want |= set(_numpy_knn(ix["q"][cv], qq, k).tolist())
    cand = sorted(want)
    costs = [O.cost64(g, m, K, tl, ix["dict"][j]) for j in cand]
    assert log[0, 2] == cand[int(np.argmin(costs))]


def test_fill_criminisi_priority_runs():
    g, m = synth.voronoi2d(40, cfg=2, seed_sub=6)
    out, mo, log, steps = O.inpaint(g, m, 5, mode=0, prio=1)
    assert mo.all() and steps > 0


def _prio_grid(name, X=16, Y=16):
    y, x = np.mgrid[0:Y, 0:X].astype(np.float64)
    if name == "quad":
        v = x * x / 256 + y / 32
    else:
        v = x / 64 + y / 32
    if name == "ramp_rgb":
        return np.stack([v + 0.25, v, v - 0.25], -1).astype(np.float32)
    return v[..., None].astype(np.float32)


def _prio_mask(name, X=16, Y=16):
    y, x = np.mgrid[0:Y, 0:X]
    unknown = {"vcol10": x >= 10, "diag14": x + y >= 14, "cols8_10": (x == 8) | (x == 10),
               "col2": (x == 2) & (y >= 4) & (y < 8)}[name]
    return (~unknown).astype(np.uint8)


def _frac(t):
    s = 1 / np.sqrt(2.0)
    neg = t.startswith("-")
    t = t.lstrip("-")
    if t == "s":
        v = s
    elif t.endswith("s/256") or t.endswith("s/64"):
        num, den = t.split("s/")
        v = float(num or 1) * s / float(den)
    elif "/" in t:
        a, b = t.split("/")
        v = float(a) / float(b)
    else:
        v = float(t)
    return -v if neg else v


def test_criminisi_priority_terms_hand_worked():
    # Each term of the fill order (Sec. I, Sec. II.G: Criminisi's priority) at
    # hand-worked pixels: the one-sided difference from the known side, a zero
    # difference when both neighbours (or the centre) are unknown, the mask
    # normal of straight and diagonal edges, the channel mean, and D(p) as the
    # isophote (not the gradient) against the normal.
    n = 0
    for line in open(os.path.join(GOLD, "criminisi_priority.txt")):
        if line.startswith("#") or not line.strip():
            continue
        gname, mname, K, cx, cy, *vals = line.strip().split(";")
        t = O.priority(_prio_grid(gname), _prio_mask(mname), int(K), (int(cx), int(cy)), prio=1)
        for key, want in zip(("C", "gx", "gy", "nx", "ny", "D"), vals):
            assert t[key] == pytest.approx(_frac(want), rel=1e-6, abs=1e-12), (line, key)
        assert t["P"] == pytest.approx(t["C"] * (t["D"] + 0.001), rel=1e-6)
        # the confidence-only priority is C(p) alone
        assert O.priority(_prio_grid(gname), _prio_mask(mname), int(K), (int(cx), int(cy)), prio=0)["P"] == t["C"]
        n += 1
    assert n >= 6


def test_criminisi_first_target_differs_from_confidence():
    # 24 x 24 ramp I = x/64 + y/32, square hole [10, 14)^2, K = 3.  Front
    # centres: top/bottom rows (x = 10..13, y = 9 / 14) and left/right columns
    # (x = 9 / 14, y = 10..13).  Confidence: 7/9 at the four ends of each side
    # (two unknown pixels in the patch), 6/9 in between.  CONFIDENCE takes the
    # lowest linear index among the 7/9 centres: (10, 9).  The data term is
    # |g_x| = 1/64 on the top and bottom sides (normal (0, -+1)) and |g_y| = 1/32
    # on the left and right sides (normal (-+1, 0)), so CRIMINISI takes the
    # lowest linear index among the left/right ends: (9, 10).  (The gradient
    # instead of the isophote would swap the two sides and pick (10, 9).)
    g = _prio_grid("ramp", 24, 24)
    m = np.ones((24, 24), np.uint8)
    m[10:14, 10:14] = 0
    _, _, log_c, _ = O.inpaint(g, m, 3, mode=0, prio=0, max_steps=1)
    _, _, log_k, _ = O.inpaint(g, m, 3, mode=0, prio=1, max_steps=1)
    assert tuple(log_c[0, :2]) == (10, 9)
    assert tuple(log_k[0, :2]) == (9, 10)
    ends = {(10, 9), (13, 9), (10, 14), (13, 14), (9, 10), (9, 13), (14, 10), (14, 13)}
    for c in ends:
        t = O.priority(g, m, 3, c, prio=1)
        assert t["C"] == pytest.approx(7 / 9, rel=1e-7)
        assert t["D"] == (1 / 32 if c[0] in (9, 14) else 1 / 64)
    for c in [(11, 9), (9, 11), (12, 14), (14, 12)]:
        assert O.priority(g, m, 3, c, prio=1)["C"] == pytest.approx(6 / 9, rel=1e-7)


def test_empty_dictionary_is_an_error():
    g = np.zeros((6, 6, 1), np.float32)
    m = np.zeros((6, 6), np.uint8)
    m[0, 0] = 1
    with pytest.raises(ValueError):
        O.inpaint(g, m, 3)
