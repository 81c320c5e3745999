"""Runs of the CPU oracle spread over host cores (test infrastructure only).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: used by ``tests/`` and
by the CPU-baseline leg of ``bench.py``.  Nothing here computes anything of the
method: every number comes from the single-threaded oracle functions of
``oracle/__init__.py``; this module only hands independent pieces of work to
worker processes and puts their results back together in order.

* the indices of a multi-index are independent (one PCA, projection, quantiser,
  key array and sort per index, Sec. II.A-C), so each worker builds one index;
* queries are independent (Fig. 1(b)-(d)), so query batches are split into
  contiguous chunks;
* full-scan targets are independent (Sec. I), likewise.

Workers are started with the ``spawn`` method: a process that has initialised
CUDA must never fork.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os
import shutil
import tempfile

import numpy as np

_W = {}  # per-worker cache: arrays loaded from the job's files


def default_workers() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def make_pool(workers: int | None = None) -> cf.ProcessPoolExecutor:
    """A spawned pool whose workers have loaded the oracle library."""
    n = workers or default_workers()
    ex = cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"), initializer=_init_worker)
    # start every worker now (so a timed region does not include start-up)
    list(ex.map(_noop, range(n)))
    return ex


def _init_worker():
    import oracle as O

    O.lib()


def _noop(i):
    return i


class Stash:
    """Arrays shared with the workers through .npy files in a private temporary
    directory (each worker maps a file once and keeps it)."""

    def __init__(self):
        self.dir = tempfile.mkdtemp(prefix="oracle_pool_")
        self.n = 0

    def put(self, a) -> str:
        if a is None:
            return None
        path = os.path.join(self.dir, f"a{self.n}.npy")
        self.n += 1
        np.save(path, np.ascontiguousarray(a))
        return path

    def close(self):
        shutil.rmtree(self.dir, ignore_errors=True)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _get(path):
    if path is None:
        return None
    if path not in _W:
        d = os.path.dirname(path)
        if _W.get("_dir") != d:  # a new job: drop the previous job's maps
            _W.clear()
            _W["_dir"] = d
        _W[path] = np.load(path, mmap_mode="r")
    return _W[path]


# ----------------------------------------------------------------------------
# one index of a multi-index (Sec. II.A-C)
# ----------------------------------------------------------------------------
def _build_curve(paths, cv, K, D, bits, sample, basis, mean, shift, curve):
    import oracle as O

    grid, dct, sub = (np.asarray(_get(p)) for p in paths)
    if basis is None:
        B, MU, EV, _ = O.pca(grid, K, dct, sub[cv], sample, D)
    else:
        B, MU, EV = basis, mean, np.full(sub.shape[1] * grid.shape[-1], np.nan)
    Y = O.project(grid, K, dct, sub[cv], B, MU, D)
    lo, sc = O.quant_params(Y, bits)
    q = O.quantise(Y, bits, lo, sc)
    k = O.keys(q, bits, shift, curve)
    sk, si = O.sort(k)
    return cv, B, MU, EV, Y, lo, sc, q, k, sk, si


def build_index(ex, grid, mask, K, C_, D, bits, frac=0.6, sample=1 << 20, shifts=None, basis=None, mean=None,
                curve=0):
    """oracle.build_index with its indices built by the workers of `ex`; the
    result is the same dictionary of arrays."""
    import oracle as O

    ndim, ext, ch = O.geometry(grid)
    dct = O.dict_extract(mask, K)
    sub = O.subsets(ndim, K, frac, C_)
    sh = None if shifts is None else np.ascontiguousarray(shifts, np.int32).reshape(C_, D)
    with Stash() as stash:
        paths = (stash.put(np.asarray(grid, np.float32)), stash.put(dct), stash.put(sub))
        futs = [ex.submit(_build_curve, paths, cv, K, D, bits, sample, None if basis is None else basis[cv],
                          None if mean is None else mean[cv], None if sh is None else sh[cv], curve)
                for cv in range(C_)]
        parts = sorted((f.result() for f in futs), key=lambda r: r[0])
    st = lambda i: np.stack([p[i] for p in parts])  # noqa: E731
    return dict(ndim=ndim, ext=ext, ch=ch, K=K, C=C_, D=D, bits=bits, dict=dct, N=len(dct), subset=sub,
                m=sub.shape[1], basis=st(1), mean=st(2), evals=st(3), proj=st(4), lo=st(5), scale=st(6), q=st(7),
                keys=st(8), skeys=st(9), sids=st(10), shifts=sh, curve=curve)


# ----------------------------------------------------------------------------
# query batches (Fig. 1(b)-(d)) and full scans (Sec. I)
# ----------------------------------------------------------------------------
_IX_ARRAYS = ("ext", "dict", "subset", "basis", "mean", "lo", "scale", "skeys", "sids", "shifts")
_IX_SCALARS = ("ndim", "ch", "K", "C", "D", "bits", "N", "m", "curve")


def _query_chunk(ixp, gp, mp_, lins, W):
    import oracle as O

    ix = {k: (None if v is None else np.asarray(_get(v))) for k, v in ixp["arrays"].items()}
    ix.update(ixp["scalars"])
    grid, mask = np.asarray(_get(gp)), np.asarray(_get(mp_))
    out = []
    for tl in lins:
        r = O.query(ix, grid, mask, int(tl), W)
        out.append((r["pick"], r["cost"], r["cand"]))
    return out


def query_batch(ex, workers, ix, grid, cur_mask, targets_lin, W):
    """oracle.query for every target -> (picks int64[Q], costs float64[Q], list of candidate arrays)."""
    with Stash() as stash:
        ixp = {"arrays": {k: stash.put(ix.get(k)) for k in _IX_ARRAYS},
               "scalars": {k: ix.get(k, 0) for k in _IX_SCALARS}}
        gp = stash.put(np.asarray(grid, np.float32))
        mp_ = stash.put(np.asarray(cur_mask, np.uint8))
        chunks = np.array_split(np.asarray(targets_lin, np.int64), max(1, 4 * workers))
        n = len(chunks)
        res = [r for part in ex.map(_query_chunk, [ixp] * n, [gp] * n, [mp_] * n, chunks, [W] * n) for r in part]
    return (np.array([r[0] for r in res], np.int64), np.array([r[1] for r in res], np.float64),
            [r[2] for r in res])


def _fullscan_chunk(gp, mp_, dp, lins, K):
    import oracle as O

    return O.fullscan(np.asarray(_get(gp)), np.asarray(_get(mp_)), K, np.asarray(_get(dp)), lins)


def fullscan(ex, workers, grid, cur_mask, K, dict_lin, targets_lin):
    """oracle.fullscan with the targets split over the workers -> (picks, costs)."""
    with Stash() as stash:
        gp = stash.put(np.asarray(grid, np.float32))
        mp_ = stash.put(np.asarray(cur_mask, np.uint8))
        dp = stash.put(np.asarray(dict_lin, np.int64))
        chunks = [c for c in np.array_split(np.asarray(targets_lin, np.int64), workers) if len(c)]
        n = len(chunks)
        res = list(ex.map(_fullscan_chunk, [gp] * n, [mp_] * n, [dp] * n, chunks, [K] * n))
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])
