"""Multi-GPU data paths of the patch search: host logic, one process per GPU.

The paper parallelises over queries and over the dictionary (Sec. II.F, on CPU
threads).  On several GPUs the two become:

* the dictionary split of the exact full scan (Sec. I): every rank owns a
  contiguous range of dictionary ids (``sfc_shard_*`` of the C-ABI); one
  all-reduce-min of each query's minimum FP32 cost (float bits: costs are >= 0,
  so the bits order like the values), the FP64 rescore of the entries inside the
  FP32 error band of that minimum on every rank, and one all-gather of
  (FP64 cost, id, FP32 cost) per query and rank, whose (FP64 cost, id) minimum is
  the pick -- the same picks and costs as the single-GPU scan;
* query sharding over a replicated index for the SFC search (Fig. 1(b)-(d)):
  every rank builds the same index (the build is deterministic) and answers a
  contiguous range of the queries; an all-gather puts the answers back in order.
  (Windows taken on a sharded sorted array would differ from the global ones, so
  the index itself is not split.)

The collective steps take the per-rank work as functions, so the same code runs
with the GPU entry points (``fullscan_dict_split``, ``query_batch_split``) and,
in the CPU tests, with stand-ins on ``gloo`` ranks.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch
import torch.distributed as dist

from . import sfc

INT64_MAX = np.iinfo(np.int64).max


def shard_bounds(n: int, shard: int, nshards: int) -> tuple[int, int]:
    """The contiguous share [lo, hi) of n items owned by shard `shard` of
    `nshards` (the rule of sfc_shard_create)."""
    return n * shard // nshards, n * (shard + 1) // nshards


def _world(group):
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def merge_shard_results(cost64: torch.Tensor, ids: torch.Tensor, cost32: torch.Tensor):
    """(R, Q) per-rank shard minima -> (pick int64[Q], cost float32[Q]): the
    (FP64 cost, id) minimum over the ranks and the FP32 cost that came with it;
    pick -1 and cost NaN where no rank holds a band entry (an invalid centre)."""
    c = torch.where(torch.isnan(cost64) | (ids < 0), torch.full_like(cost64, float("inf")), cost64)
    best = c.min(dim=0).values
    cand = (c == best.unsqueeze(0)) & (ids >= 0)
    idm = torch.where(cand, ids, torch.full_like(ids, INT64_MAX))
    pick = idm.min(dim=0).values
    r = (idm == pick.unsqueeze(0)).to(torch.int64).argmax(dim=0)
    cost = cost32.gather(0, r.unsqueeze(0)).squeeze(0)
    none = pick == INT64_MAX
    pick = torch.where(none, torch.full_like(pick, -1), pick)
    cost = torch.where(none, torch.full_like(cost, float("nan")), cost)
    return pick, cost


def split_fullscan(scan_fn, band_fn, group=None):
    """The exchange of the dictionary split.  scan_fn() -> int32 [Q] (the
    rank's minimum FP32 cost per query, as float bits); band_fn(gmin) ->
    (float64 [Q], int64 [Q], float32 [Q]) for the global minimum gmin.
    Returns (pick, cost) on every rank."""
    rank, world = _world(group)
    m = scan_fn()
    if world > 1:
        dist.all_reduce(m, op=dist.ReduceOp.MIN, group=group)
    c64, ids, c32 = band_fn(m)
    if world == 1:
        return merge_shard_results(c64.unsqueeze(0), ids.unsqueeze(0), c32.unsqueeze(0))
    parts = []
    for t in (c64, ids, c32):
        out = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(out, t, group=group)
        parts.append(torch.stack(out))
    return merge_shard_results(*parts)


def split_queries(query_fn, Q: int, group=None):
    """Query sharding: query_fn(q0, q1) -> (pick int64 [q1-q0], cost float32
    [q1-q0]) for the rank's range; returns every query's (pick, cost) in order
    on every rank."""
    rank, world = _world(group)
    q0, q1 = shard_bounds(Q, rank, world)
    pick, cost = query_fn(q0, q1)
    if world == 1:
        return pick, cost
    cap = -(-Q // world)  # the largest share
    pp = torch.full((cap,), -1, dtype=torch.int64, device=pick.device)
    cc = torch.full((cap,), float("nan"), dtype=torch.float32, device=cost.device)
    pp[: q1 - q0] = pick
    cc[: q1 - q0] = cost
    outp = [torch.empty_like(pp) for _ in range(world)]
    outc = [torch.empty_like(cc) for _ in range(world)]
    dist.all_gather(outp, pp, group=group)
    dist.all_gather(outc, cc, group=group)
    picks, costs = [], []
    for r in range(world):
        a, b = shard_bounds(Q, r, world)
        picks.append(outp[r][: b - a])
        costs.append(outc[r][: b - a])
    return torch.cat(picks), torch.cat(costs)


# ----------------------------------------------------------------------------
# the GPU entry points
# ----------------------------------------------------------------------------
class Shard:
    """Owner of an sfc_shard: one rank's share of a full scan's dictionary."""

    def __init__(self, grid, dict_mask, cur_mask, centres, K, shard, nshards, **params):
        L = sfc.lib()
        self.grid = sfc._dev(grid, torch.float32)
        self.dict_mask = sfc._dev(dict_mask, torch.uint8)
        self.cur_mask = sfc._dev(cur_mask, torch.uint8)
        self.centres = sfc._dev(centres, torch.int32)
        self.Q = self.centres.shape[0]
        P = sfc.Params(K=K, **params)
        g = sfc.make_grid(self.grid)
        h = C.c_void_p()
        sfc._check(L.sfc_shard_create(sfc._ptr(self.grid), sfc._ptr(self.dict_mask), sfc._ptr(self.cur_mask),
                                      C.byref(g), C.byref(P.p), sfc._ptr(self.centres), self.Q, shard, nshards,
                                      sfc._stream(), C.byref(h)), "sfc_shard_create")
        self.h = h
        N, j0, j1 = C.c_int64(), C.c_int64(), C.c_int64()
        sfc._check(L.sfc_shard_range(self.h, C.byref(N), C.byref(j0), C.byref(j1)), "sfc_shard_range")
        self.N, self.j0, self.j1 = N.value, j0.value, j1.value

    def scan(self) -> torch.Tensor:
        m = torch.empty(self.Q, dtype=torch.int32, device=self.grid.device)
        sfc._check(sfc.lib().sfc_shard_scan(self.h, sfc._ptr(m), sfc._stream()), "sfc_shard_scan")
        return m

    def band(self, gmin: torch.Tensor):
        dev = self.grid.device
        c64 = torch.empty(self.Q, dtype=torch.float64, device=dev)
        ids = torch.empty(self.Q, dtype=torch.int64, device=dev)
        c32 = torch.empty(self.Q, dtype=torch.float32, device=dev)
        sfc._check(sfc.lib().sfc_shard_band(self.h, sfc._ptr(gmin), sfc._ptr(c64), sfc._ptr(ids), sfc._ptr(c32),
                                            sfc._stream()), "sfc_shard_band")
        return c64, ids, c32

    def close(self):
        if self.h:
            sfc.lib().sfc_shard_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def fullscan_dict_split(grid, dict_mask, cur_mask, centres, K, group=None, **params):
    """fullscan_query_batch with the dictionary shared out among the ranks of
    `group` (one GPU each): this rank scans its share; returns every query's
    (pick, cost) on every rank."""
    rank, world = _world(group)
    sh = Shard(grid, dict_mask, cur_mask, centres, K, rank, world, **params)
    try:
        return split_fullscan(sh.scan, sh.band, group)
    finally:
        sh.close()


def query_batch_split(ix, grid, cur_mask, centres, group=None):
    """sfc_query_batch with the queries shared out among the ranks of `group`,
    each holding the same index; returns every query's (pick, cost)."""
    centres = sfc._dev(centres, torch.int32)

    def run(q0, q1):
        return sfc.sfc_query_batch(ix, grid, cur_mask, centres[q0:q1].contiguous())

    return split_queries(run, centres.shape[0], group)
