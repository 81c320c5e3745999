"""The parameter search's selection rule and its argument checks, on the host
(no GPU): sfc_tune_select and sfc_autotune's refusals before any device work."""
import ctypes as C
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1712_06326_gb300 import sfc

    return sfc


def test_fastest_within_the_error_bound(S):
    ms = [5.0, 2.0, 3.0, 1.0]
    ae = [0.001, 0.02, 0.005, 0.5]
    assert S.sfc_tune_select(ms, ae, 0.01) == 2
    assert S.sfc_tune_select(ms, ae, 1.0) == 3
    assert S.sfc_tune_select(ms, ae, 0.001) == 0


def test_ties_go_to_list_order(S):
    assert S.sfc_tune_select([2.0, 1.0, 1.0], [0.0, 0.0, 0.0], 0.01) == 1
    # none within the bound: least error, then the faster, then list order
    assert S.sfc_tune_select([3.0, 2.0, 2.0, 1.0], [0.2, 0.1, 0.1, 0.3], 0.01) == 1
    assert S.sfc_tune_select([3.0, 1.0], [0.1, 0.1], 0.0) == 1


def test_nan_counts_as_infinity(S):
    assert S.sfc_tune_select([math.nan, 2.0], [0.0, 0.0], 0.01) == 1
    assert S.sfc_tune_select([1.0, 2.0], [math.nan, 0.5], 0.01) == 1
    assert S.sfc_tune_select([1.0], [math.nan], 0.01) == 0


def test_empty_is_minus_one(S):
    L = S.lib()
    assert L.sfc_tune_select(0, None, None, 0.01) == -1


def test_autotune_refuses_bad_specs_on_the_host(S):
    L = S.lib()
    g = S.sfc_grid()
    g.ndim, g.ch = 2, 3
    g.ext[0], g.ext[1], g.ext[2] = 64, 64, 1
    p = S.sfc_params()
    L.sfc_params_default(C.byref(p))
    best = S.sfc_params()
    fake = C.c_void_p(256)  # never dereferenced: every check below fails first
    lists = [np.array(v, np.int32) for v in ([4, 8], [6, 8], [16, 64])]

    def spec(**kw):
        s = S.sfc_tune_spec()
        s.curves, s.n_curves = lists[0].ctypes.data_as(C.c_void_p), 2
        s.dims, s.n_dims = lists[1].ctypes.data_as(C.c_void_p), 2
        s.windows, s.n_windows = lists[2].ctypes.data_as(C.c_void_p), 2
        s.sample, s.reps, s.objective, s.ae_max = 64, 1, S.SFC_TUNE_STEP, 0.01
        for k, v in kw.items():
            setattr(s, k, v)
        return s

    def call(sp, q=10, params=p):
        return L.sfc_autotune(fake, fake, C.byref(g), C.byref(params), fake, q, C.byref(sp), C.byref(best), None,
                              None, None)

    for bad in (dict(n_curves=0), dict(sample=0), dict(reps=0), dict(reps=101), dict(objective=7),
                dict(ae_max=-1.0), dict(ae_max=math.nan), dict(dims=None)):
        assert call(spec(**bad)) == S.SFC_EINVAL, bad
        assert "sfc_autotune" in L.sfc_last_error().decode()
    assert call(spec(), q=0) == S.SFC_EINVAL
    many = np.arange(1, 20, dtype=np.int32)
    big = spec(windows=many.ctypes.data_as(C.c_void_p), n_windows=19)
    big.curves, big.n_curves = many.ctypes.data_as(C.c_void_p), 19
    big.dims, big.n_dims = many.ctypes.data_as(C.c_void_p), 19
    assert call(big) == S.SFC_EINVAL and "4096" in L.sfc_last_error().decode()
    sh = np.zeros(64, np.int32)
    p2 = S.sfc_params()
    L.sfc_params_default(C.byref(p2))
    p2.shifts = sh.ctypes.data_as(C.c_void_p)
    assert call(spec(), params=p2) == S.SFC_EINVAL and "shifts" in L.sfc_last_error().decode()
