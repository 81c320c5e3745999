"""Failure paths that actually run (needs a GB300), without faulting the GPU.

* A bounded device wait made to run out: the radix sort's decoupled look-back
  (each sort tile polls its predecessors' published digit counts) is switched
  to poll a word nothing writes, with a short poll limit.  Every tile after the
  first gives up, flags the library's status word and carries on with its
  writes kept inside the output arrays; the build returns, sfc_status() reports
  SFC_ETIMEOUT, and the same context then builds and queries correctly.  (The
  tensor-core GEMM's mbarrier waits are not shortened for a test: a CTA that
  gave up with bulk copies in flight would not be a safe thing to run.)
* Device allocations made to fail one at a time on the host: every entry point
  that allocates returns SFC_ENOMEM at each of its allocations and gives back
  everything it had taken (the library pool's used bytes return to where they
  were).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1712_06326_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1712_06326_gb300 import sfc

    torch.cuda.set_device(0)
    sfc.sfc_status()
    yield sfc
    sfc.sfc_debug_lookback(0, False)
    sfc.sfc_debug_sort(False, 0)
    sfc.sfc_debug_fail_alloc(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_queries_match_oracle(S, g, m, t, K, C_, D, bits, W):
    ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0)
    ex = S.sfc_index_export(ix)
    pk, _ = S.sfc_query_batch(ix, dev(g), dev(m), dev(t))
    ix.close()
    oix = O.build_index(g, m, K, C_, D, bits, basis=ex["basis"], mean=ex["mean"])
    assert np.array_equal(oix["skeys"], ex["skeys"]) and np.array_equal(oix["sids"], ex["sids"])
    lin = O.centres_to_lin(t, O.geometry(g)[1])
    pk = pk.cpu().numpy()
    for i, tl in enumerate(lin):
        assert pk[i] == O.query(oix, g, m, tl, W)["pick"]


def test_sort_lookback_timeout_is_reported_and_the_gpu_recovers(S):
    g, m = synth.voronoi2d(256, cfg=2, seed_sub=4)
    t = synth.front_targets(m, 9, cap=32, cfg=2)
    K, C_, D, bits, W = 9, 4, 6, 10, 32
    assert len(O.dict_extract(m, K)) > 8 * 3072  # several sort tiles per index
    assert S.sfc_status() == 0
    S.sfc_debug_sort(True, 0)  # the LSD radix sort (dictionaries this small take the sample sort)
    S.sfc_debug_lookback(2000, True)
    try:
        ix = S.sfc_index_build(dev(g), dev(m), K=K, curves=C_, dims=D, bits=bits, window=W, pca_sample=0)
        assert S.sfc_status() == S.SFC_ETIMEOUT
        ix.close()
    finally:
        S.sfc_debug_lookback(0, False)
        S.sfc_debug_sort(False, 0)
    assert S.sfc_status() == 0  # read and cleared
    # the same context: a normal build sorts correctly and answers like the oracle
    check_queries_match_oracle(S, g, m, t, K, C_, D, bits, W)
    assert S.sfc_status() == 0


def count_allocs(S, fn):
    a0 = S.sfc_debug_alloc_count()
    fn()
    torch.cuda.synchronize()
    return S.sfc_debug_alloc_count() - a0


def every_allocation_fails_cleanly(S, fn, what):
    n = count_allocs(S, fn)
    assert n > 0, what
    base = S.sfc_debug_pool_used()
    for k in range(1, n + 1):
        S.sfc_debug_fail_alloc(k)
        try:
            with pytest.raises(RuntimeError, match=r"\(-2\)"):
                fn()
        finally:
            S.sfc_debug_fail_alloc(0)
        assert S.sfc_debug_pool_used() == base, f"{what}: allocation {k} of {n} left memory behind"
    return n


def test_allocation_failures_return_enomem_and_release_everything(S):
    g, m = synth.voronoi2d(96, cfg=2, seed_sub=5)
    t = np.concatenate([synth.front_targets(m, 7, cap=20, cfg=2), synth.random_targets(m, 7, 12, cfg=2)])
    gd, md, td = dev(g), dev(m), dev(t)
    prm = dict(K=7, curves=4, dims=5, bits=10, window=24, pca_sample=0)

    def build():
        S.sfc_index_build(gd, md, **prm).close()

    def build_knn():
        S.sfc_index_build(gd, md, **dict(prm, knn=16)).close()

    def fullscan():
        S.fullscan_query_batch(gd, md, md, td, K=7)

    def fullscan_tc():
        S.fullscan_query_batch(gd, md, md, td, K=7, precision=S.SFC_FP16)

    def fill():
        S.inpaint_run(gd.clone(), md.clone(), mode=S.SFC_MODE_FULLSCAN, max_steps=3, K=7)

    def fill_sfc():
        S.inpaint_run(gd.clone(), md.clone(), mode=S.SFC_MODE_SFC, max_steps=3, **prm)

    counts = {}
    for fn in (build, build_knn, fullscan, fullscan_tc, fill, fill_sfc):
        counts[fn.__name__] = every_allocation_fails_cleanly(S, fn, fn.__name__)
    assert counts["build"] >= 10
    assert S.sfc_status() == 0
    # nothing left armed: the library still answers like the oracle
    fp, _ = S.fullscan_query_batch(gd, md, md, td, K=7)
    op, _ = O.fullscan(g, m, 7, O.dict_extract(m, 7), O.centres_to_lin(t, O.geometry(g)[1]))
    assert np.array_equal(fp.cpu().numpy(), op)
