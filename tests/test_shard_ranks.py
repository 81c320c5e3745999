"""The multi-GPU data paths' host logic on CPU ranks (gloo, world sizes 1-3):
the dictionary split of the full scan and query sharding over a replicated
index (paper_1712_06326_gb300/shard.py).  The per-rank device work is played
by the oracle: the shard scan's FP32 costs are the oracle's exact costs
rounded to FP32 (within the FP32 error band the library uses), its band pass
rescoring with the oracle's exact FP64 cost.  Bars: the split answers equal the
single-rank answers and the oracle's brute-force picks, bit for bit, with
uneven and empty shares."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1712_06326_gb300 import shard as SH
from paper_1712_06326_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case(tiny=False):
    if tiny:  # a dictionary smaller than the rank count: empty shares
        g = np.random.default_rng(3).random((8, 8, 1)).astype(np.float32)
        m = np.zeros((8, 8), np.uint8)
        m[0:3, 0:4] = 1  # two fully known 3x3 patches
        t = np.array([[4, 4], [5, 5]], np.int32)
        return g, m, t, 3
    g, m = synth.voronoi2d(48, cfg=2, seed_sub=9)
    t = np.concatenate([synth.front_targets(m, 5, cap=12, cfg=2), synth.random_targets(m, 5, 5, cfg=2)])
    # an exact tie across shares: the lowest id must win
    g[30:35, 40:45] = g[2:7, 2:7]
    return g, m, t.astype(np.int32), 5


def _band_limit32(m32, n):
    # the FP32 error band of the scan: m (1 + 3 (n + 8) 2^-24) rounded up
    return np.nextafter(np.float32(m32 * (1.0 + 3.0 * (n + 8) * 2.0 ** -24)), np.float32(np.inf))


def _stand_in(g, m, t, K, rank, world):
    d = O.dict_extract(m, K)
    lin = O.centres_to_lin(t, O.geometry(g)[1])
    j0, j1 = SH.shard_bounds(len(d), rank, world)
    n = K * K * g.shape[2]
    cost64 = np.array([[O.cost64(g, m, K, tl, d[j]) for j in range(j0, j1)] for tl in lin]).reshape(len(lin), -1)
    cost32 = cost64.astype(np.float32)

    def scan():
        mins = cost32.min(axis=1) if j1 > j0 else np.full(len(lin), np.inf, np.float32)
        return torch.from_numpy(mins.astype(np.float32).view(np.int32).copy())

    def band(gmin):
        gm = gmin.numpy().view(np.float32)
        c64 = np.full(len(lin), np.inf)
        ids = np.full(len(lin), -1, np.int64)
        c32 = np.full(len(lin), np.inf, np.float32)
        for q in range(len(lin)):
            T = _band_limit32(gm[q], n)
            for k in range(j1 - j0):
                if cost32[q, k] <= T and (cost64[q, k], j0 + k) < (c64[q], ids[q] if ids[q] >= 0 else 2 ** 62):
                    c64[q], ids[q], c32[q] = cost64[q, k], j0 + k, cost32[q, k]
        return torch.from_numpy(c64), torch.from_numpy(ids), torch.from_numpy(c32)

    return scan, band, d, lin


def _run(rank, world, port, out, tiny):
    if world > 1:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=world)
    g, m, t, K = _case(tiny)
    scan, band, d, lin = _stand_in(g, m, t, K, rank, world)
    pick, cost = SH.split_fullscan(scan, band)
    # query sharding: each rank answers its share of the queries on the same index
    ix = O.build_index(g, m, K, 2, 3, 8)

    def qfn(q0, q1):
        rs = [O.query(ix, g, m, tl, 16) for tl in lin[q0:q1]]
        return (torch.tensor([r["pick"] for r in rs], dtype=torch.int64),
                torch.tensor([r["cost"] for r in rs], dtype=torch.float32))

    qp, qc = SH.split_queries(qfn, len(lin))
    out[(world, rank)] = (pick.numpy(), cost.numpy(), qp.numpy(), qc.numpy())
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def _launch(world, tiny=False):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_run, args=(r, world, port, out, tiny)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    return dict(out)


def test_dictionary_split_and_query_sharding_equal_one_rank():
    ref = {}
    _run(0, 1, 0, ref, False)
    p1, c1, q1, qc1 = ref[(1, 0)]
    g, m, t, K = _case()
    op, oc = O.fullscan(g, m, K, O.dict_extract(m, K), O.centres_to_lin(t, O.geometry(g)[1]))
    assert np.array_equal(p1, op)  # the single-rank stand-in reaches the exact picks
    for world in (2, 3):
        res = _launch(world)
        for r in range(world):
            p, c, q, qc = res[(world, r)]
            assert np.array_equal(p, p1) and np.array_equal(c.view(np.int32), c1.view(np.int32))
            assert np.array_equal(q, q1) and np.array_equal(qc.view(np.int32), qc1.view(np.int32))


def test_empty_shares():
    res = _launch(3, tiny=True)  # 2 dictionary entries over 3 ranks, 2 queries
    ref = {}
    _run(0, 1, 0, ref, True)
    for r in range(3):
        assert np.array_equal(res[(3, r)][0], ref[(1, 0)][0])
    assert all(p >= 0 for p in ref[(1, 0)][0])


def test_merge_rule():
    # (cost64, id) minimum over ranks; NaN / -1 entries never win; all-empty -> -1, NaN
    c64 = torch.tensor([[2.0, np.inf, np.nan], [1.0, 3.0, np.nan], [1.0, 3.0, np.nan]], dtype=torch.float64)
    ids = torch.tensor([[4, -1, -1], [9, 7, -1], [8, 6, -1]], dtype=torch.int64)
    c32 = torch.tensor([[2.0, np.inf, np.nan], [1.5, 3.5, np.nan], [1.25, 3.25, np.nan]], dtype=torch.float32)
    p, c = SH.merge_shard_results(c64, ids, c32)
    assert p.tolist() == [8, 6, -1]
    assert c[0].item() == 1.25 and c[1].item() == 3.25 and np.isnan(c[2].item())
