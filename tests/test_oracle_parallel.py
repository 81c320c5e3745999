"""The oracle's multi-process harness (oracle/parallel.py) returns exactly what
the single-threaded oracle returns: it only splits independent work (indices,
queries, full-scan targets) over spawned workers.  No GPU."""
import numpy as np
import pytest

import oracle as O
from oracle import parallel as OP
from paper_1712_06326_gb300 import synth


@pytest.fixture(scope="module")
def pool():
    ex = OP.make_pool(2)
    yield ex
    ex.shutdown()


def test_parallel_index_query_and_fullscan_equal_serial(pool):
    g, m = synth.voronoi2d(72, cfg=2, seed_sub=3)
    K, C_, D, bits, W = 7, 4, 5, 10, 24
    ref = O.build_index(g, m, K, C_, D, bits, sample=500)
    par = OP.build_index(pool, g, m, K, C_, D, bits, sample=500)
    for k in ("dict", "subset", "basis", "mean", "proj", "lo", "scale", "q", "keys", "skeys", "sids"):
        assert np.array_equal(ref[k], par[k]), k
    assert np.allclose(ref["evals"], par["evals"], rtol=0, atol=0, equal_nan=True)
    t = synth.front_targets(m, K, cap=50, cfg=2)
    lin = O.centres_to_lin(t, O.geometry(g)[1])
    pk, cs, cand = OP.query_batch(pool, 2, par, g, m, lin, W)
    for i, tl in enumerate(lin):
        r = O.query(ref, g, m, tl, W)
        assert pk[i] == r["pick"] and cs[i] == r["cost"] and np.array_equal(cand[i], r["cand"])
    fp, fc = OP.fullscan(pool, 2, g, m, K, ref["dict"], lin[:9])
    sp, sc = O.fullscan(g, m, K, ref["dict"], lin[:9])
    assert np.array_equal(fp, sp) and np.array_equal(fc, sc)
