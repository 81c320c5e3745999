"""fullscan_query_batch_static: the full scan for callers that cannot allocate
device memory (their host framework's allocator owns the device memory, or they
cannot afford the synchronisation an allocation may cause).  It keeps all scratch
in the library's fixed 16 MiB static device array.

Checked through the C-ABI against fullscan_query_batch, which allocates its
scratch: picks and costs must be identical (the exact-cost tolerance of the
other tests: bit-exact), on two different calls in a row, so the second call
also proves that leftovers of the first in the shared array do not leak into it.
This file is collected last on purpose.
"""
import ctypes as C

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
    return sfc


def _call_static(S, g, m, t, K, w=None, norm=0):
    gd = torch.from_numpy(np.ascontiguousarray(g)).cuda()
    md = torch.from_numpy(np.ascontiguousarray(m)).cuda()
    td = torch.from_numpy(np.ascontiguousarray(t, np.int32)).cuda()
    Q = td.shape[0]
    pick = torch.full((Q,), -7, dtype=torch.int64, device="cuda")
    cost = torch.full((Q,), -7.0, dtype=torch.float32, device="cuda")
    P = S.Params(K=K, ch_weights=w, cost=norm)
    geo = S.make_grid(gd)
    rc = S.lib().fullscan_query_batch_static(C.c_void_p(gd.data_ptr()), C.c_void_p(md.data_ptr()),
                                             C.c_void_p(md.data_ptr()), C.byref(geo), C.byref(P.p),
                                             C.c_void_p(td.data_ptr()), Q, C.c_void_p(pick.data_ptr()),
                                             C.c_void_p(cost.data_ptr()),
                                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, S.lib().sfc_last_error()
    torch.cuda.synchronize()
    return pick.cpu().numpy(), cost.cpu().numpy()


def test_static_scratch_full_scan_matches_allocating_entry_point(S):
    g1, m1 = synth.sines2d(128)
    t1 = synth.front_targets(m1, 9)
    g2, m2 = synth.voronoi2d(96, cfg=2, seed_sub=2)
    t2 = np.concatenate([synth.front_targets(m2, 7, cap=40, cfg=2), synth.random_targets(m2, 7, 24, cfg=2)])
    w2 = np.array([1.0, 2.0, 0.5], np.float32)
    L1 = S.SFC_COST_L1
    # calls in a row on different grids and costs (L2, weighted L2, L1,
    # weighted L1), then the first again
    cases = [(g1, m1, t1, 9, None, 0), (g2, m2, t2, 7, w2, 0), (g1, m1, t1, 9, None, L1), (g2, m2, t2, 7, w2, L1),
             (g1, m1, t1, 9, None, 0)]
    S.sfc_status()  # the status word is process-wide: drop flags left by earlier calls
    for g, m, t, K, w, norm in cases:
        sp, sc = _call_static(S, g, m, t, K, w, norm)
        rp, rc = S.fullscan_query_batch(torch.from_numpy(g).cuda(), torch.from_numpy(m).cuda(),
                                        torch.from_numpy(m).cuda(), torch.from_numpy(t).cuda(), K=K, ch_weights=w,
                                        norm=norm)
        assert np.array_equal(sp, rp.cpu().numpy())
        assert np.array_equal(sc, rc.cpu().numpy())
        assert np.all(sp >= 0)
    assert S.sfc_status() == 0


def test_static_scratch_rejects_oversized_calls(S):
    g = np.zeros((2048, 2048, 1), np.float32)
    m = np.ones((2048, 2048), np.uint8)
    t = np.array([[100, 100]], np.int32)
    gd, md, td = (torch.from_numpy(a).cuda() for a in (g, m, t))
    pick = torch.empty(1, dtype=torch.int64, device="cuda")
    cost = torch.empty(1, dtype=torch.float32, device="cuda")
    P = S.Params(K=9)
    geo = S.make_grid(gd)
    rc = S.lib().fullscan_query_batch_static(C.c_void_p(gd.data_ptr()), C.c_void_p(md.data_ptr()),
                                             C.c_void_p(md.data_ptr()), C.byref(geo), C.byref(P.p),
                                             C.c_void_p(td.data_ptr()), 1, C.c_void_p(pick.data_ptr()),
                                             C.c_void_p(cost.data_ptr()), None)
    assert rc == S.SFC_EINVAL
    assert b"scratch" in S.lib().sfc_last_error()
    # a batch too large for the array is refused before any offset is formed
    rc = S.lib().fullscan_query_batch_static(C.c_void_p(gd.data_ptr()), C.c_void_p(md.data_ptr()),
                                             C.c_void_p(md.data_ptr()), C.byref(geo), C.byref(P.p),
                                             C.c_void_p(td.data_ptr()), 1 << 40, C.c_void_p(pick.data_ptr()),
                                             C.c_void_p(cost.data_ptr()), None)
    assert rc == S.SFC_EINVAL
    # the precision checks of fullscan_query_batch
    for prec, norm, want in ((7, 0, S.SFC_EUNSUPPORTED), (S.SFC_FP16, S.SFC_COST_L1, S.SFC_EUNSUPPORTED)):
        P2 = S.Params(K=9, precision=prec, cost=norm)
        rc = S.lib().fullscan_query_batch_static(C.c_void_p(gd.data_ptr()), C.c_void_p(md.data_ptr()),
                                                 C.c_void_p(md.data_ptr()), C.byref(geo), C.byref(P2.p),
                                                 C.c_void_p(td.data_ptr()), 1, C.c_void_p(pick.data_ptr()),
                                                 C.c_void_p(cost.data_ptr()), None)
        assert rc == want
