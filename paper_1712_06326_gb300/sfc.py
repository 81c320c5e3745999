"""Python binding of libsfc (include/sfc.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes device
pointers of torch CUDA tensors plus the current CUDA stream.  All computation
happens in the CUDA kernels of libsfc; there is no fallback path: if the
library is missing or a call fails, a RuntimeError is raised.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfc.so")

SFC_OK, SFC_EINVAL, SFC_ENOMEM, SFC_ECUDA, SFC_ETIMEOUT, SFC_EUNSUPPORTED, SFC_EDEVICE, SFC_ENOCONV = (
    0, -1, -2, -3, -4, -5, -6, -7)
SFC_SELECT_ALL, SFC_SELECT_BEST = 0, 1
SFC_FP32, SFC_BF16, SFC_FP16 = 0, 1, 2
SFC_PRIO_CONFIDENCE, SFC_PRIO_CRIMINISI = 0, 1
SFC_MODE_FULLSCAN, SFC_MODE_SFC = 0, 1
SFC_CURVE_MORTON, SFC_CURVE_HILBERT = 0, 1
SFC_COST_L2, SFC_COST_L1 = 0, 1
SFC_TUNE_STEP, SFC_TUNE_QUERY = 0, 1

EXPORTS = ["sfc_params_default", "sfc_index_build", "sfc_index_destroy", "sfc_index_info", "sfc_index_export",
           "sfc_query_batch", "sfc_query_candidates", "fullscan_query_batch", "fullscan_query_batch_static",
           "sfc_tc_prescores", "inpaint_run", "sfc_status", "sfc_launch_count", "sfc_trace", "sfc_trace_read", "sfc_trace_tc_read",
           "sfc_last_error", "sfc_index_save", "sfc_index_load", "sfc_index_params", "sfc_query_batch_dict",
           "sfc_multi_create", "sfc_multi_query", "sfc_multi_destroy", "sfc_autotune", "sfc_tune_select", "sfc_trace_eig_read",
           "sfc_debug_fail_alloc", "sfc_debug_alloc_count", "sfc_debug_pool_used", "sfc_debug_lookback", "sfc_debug_sort",
           "sfc_shard_create", "sfc_shard_range", "sfc_shard_scan", "sfc_shard_band", "sfc_shard_destroy",
           "sfc_trace_proj_read", "inpaint_run_multi", "sfc_tune_tiles", "sfc_tile_shape"]
TRACE_PHASES = ("dictionary", "moments", "eigen", "finalize", "project_keys", "sort")


class sfc_grid(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("ch", C.c_int32), ("ext", C.c_int64 * 3)]


class sfc_tune_spec(C.Structure):
    _fields_ = [("curves", C.c_void_p), ("n_curves", C.c_int32), ("dims", C.c_void_p), ("n_dims", C.c_int32),
                ("windows", C.c_void_p), ("n_windows", C.c_int32), ("sample", C.c_int64), ("reps", C.c_int32),
                ("objective", C.c_int32), ("ae_max", C.c_double)]


class sfc_params(C.Structure):
    _fields_ = [("K", C.c_int32), ("curves", C.c_int32), ("dims", C.c_int32), ("bits", C.c_int32),
                ("window", C.c_int32), ("subset_frac", C.c_float), ("shifts", C.c_void_p),
                ("ch_weights", C.c_void_p), ("basis", C.c_void_p), ("mean", C.c_void_p), ("select", C.c_int32),
                ("precision", C.c_int32), ("pca_sample", C.c_int64), ("priority", C.c_int32),
                ("keep_intermediates", C.c_int32), ("knn", C.c_int32), ("curve", C.c_int32),
                ("cost", C.c_int32)]


_lib = None


def lib():
    """Load libsfc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsfc.so not found at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.sfc_params_default.argtypes = [C.POINTER(sfc_params)]
        L.sfc_params_default.restype = None
        L.sfc_index_build.argtypes = [vp, vp, C.POINTER(sfc_grid), C.POINTER(sfc_params), vp, C.POINTER(vp)]
        L.sfc_index_destroy.argtypes = [vp]
        L.sfc_index_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32)]
        L.sfc_index_export.argtypes = [vp] * 12
        L.sfc_query_batch.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp]
        L.sfc_index_save.argtypes = [vp, C.c_char_p]
        L.sfc_index_params.argtypes = [vp, C.POINTER(sfc_params), C.POINTER(sfc_grid)]
        L.sfc_multi_create.argtypes = [vp, vp, vp, C.c_int32, vp, C.POINTER(vp)]
        L.sfc_multi_query.argtypes = [vp, vp, vp, i64, vp, vp, vp]
        L.sfc_multi_destroy.argtypes = [vp]
        L.sfc_index_load.argtypes = [C.c_char_p, vp, C.POINTER(vp)]
        L.sfc_query_batch_dict.argtypes = [vp, vp, vp, vp, C.POINTER(sfc_grid), vp, i64, vp, vp, vp]
        L.sfc_query_candidates.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp, vp]
        L.fullscan_query_batch.argtypes = [vp, vp, vp, C.POINTER(sfc_grid), C.POINTER(sfc_params), vp, i64, vp, vp,
                                           vp]
        L.fullscan_query_batch_static.argtypes = list(L.fullscan_query_batch.argtypes)
        L.sfc_tc_prescores.argtypes = [vp, vp, vp, C.POINTER(sfc_grid), C.POINTER(sfc_params), vp, i64, vp, vp,
                                       C.POINTER(i64), vp]
        L.inpaint_run.argtypes = [vp, vp, C.POINTER(sfc_grid), C.POINTER(sfc_params), i32, i64, vp,
                                  C.POINTER(i64), vp]
        L.inpaint_run_multi.argtypes = [vp, vp, vp, i32, C.POINTER(sfc_params), i64, vp, vp, vp]
        L.inpaint_run_multi.restype = C.c_int
        L.sfc_tune_tiles.argtypes = [vp, vp, vp, C.POINTER(sfc_grid), C.POINTER(sfc_params), vp, i64, i32, vp, vp,
                                     vp]
        L.sfc_tune_tiles.restype = C.c_int
        L.sfc_tile_shape.argtypes = [i32]
        L.sfc_tile_shape.restype = C.c_int32
        L.sfc_autotune.argtypes = [vp, vp, C.POINTER(sfc_grid), C.POINTER(sfc_params), vp, i64,
                                   C.POINTER(sfc_tune_spec), C.POINTER(sfc_params), vp, C.POINTER(i32), vp]
        L.sfc_tune_select.argtypes = [i32, vp, vp, C.c_double]
        L.sfc_tune_select.restype = C.c_int32
        L.sfc_status.argtypes = [vp]
        L.sfc_last_error.restype = C.c_char_p
        L.sfc_launch_count.restype = C.c_uint64
        L.sfc_launch_count.argtypes = []
        L.sfc_trace.argtypes = [C.c_int]
        L.sfc_trace.restype = C.c_int
        L.sfc_trace_read.argtypes = [vp, vp, vp]
        L.sfc_trace_read.restype = C.c_int
        L.sfc_trace_eig_read.argtypes = [vp, vp]
        L.sfc_trace_eig_read.restype = C.c_int
        L.sfc_trace_tc_read.argtypes = [vp, vp, vp]
        L.sfc_trace_tc_read.restype = C.c_int
        L.sfc_trace_proj_read.argtypes = [vp, vp, vp, vp]
        L.sfc_trace_proj_read.restype = C.c_int
        L.sfc_debug_fail_alloc.argtypes = [i64]
        L.sfc_debug_fail_alloc.restype = C.c_int
        L.sfc_debug_alloc_count.argtypes = []
        L.sfc_debug_alloc_count.restype = i64
        L.sfc_debug_pool_used.argtypes = [vp]
        L.sfc_debug_pool_used.restype = C.c_int
        L.sfc_debug_lookback.argtypes = [i64, i32]
        L.sfc_debug_lookback.restype = C.c_int
        L.sfc_debug_sort.argtypes = [i32, i32]
        L.sfc_debug_sort.restype = C.c_int
        L.sfc_shard_create.argtypes = [vp, vp, vp, C.POINTER(sfc_grid), C.POINTER(sfc_params), vp, i64, i32, i32, vp,
                                       C.POINTER(vp)]
        L.sfc_shard_range.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
        L.sfc_shard_scan.argtypes = [vp, vp, vp]
        L.sfc_shard_band.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sfc_shard_destroy.argtypes = [vp]
        for name in ["sfc_shard_create", "sfc_shard_range", "sfc_shard_scan", "sfc_shard_band", "sfc_shard_destroy"]:
            getattr(L, name).restype = C.c_int
        for name in ["sfc_index_build", "sfc_index_destroy", "sfc_index_info", "sfc_index_export",
                     "sfc_query_batch", "sfc_query_candidates", "fullscan_query_batch", "fullscan_query_batch_static",
                     "sfc_tc_prescores", "inpaint_run", "sfc_status", "sfc_index_save", "sfc_index_load",
                     "sfc_index_params", "sfc_query_batch_dict", "sfc_multi_create", "sfc_multi_query",
                     "sfc_multi_destroy", "sfc_autotune"]:
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != SFC_OK:
        msg = lib().sfc_last_error().decode()
        raise RuntimeError(f"{what} failed ({rc}): {msg}")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, dtype) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.ascontiguousarray(t))
    if not t.is_cuda:
        t = t.to("cuda")
    return t.to(dtype).contiguous()


def make_grid(grid: torch.Tensor) -> sfc_grid:
    """Geometry of a grid tensor laid out (Y, X, ch) or (Z, Y, X, ch)."""
    g = sfc_grid()
    if grid.dim() == 3:
        Y, X, ch = grid.shape
        g.ndim, g.ch = 2, ch
        g.ext[0], g.ext[1], g.ext[2] = X, Y, 1
    elif grid.dim() == 4:
        Z, Y, X, ch = grid.shape
        g.ndim, g.ch = 3, ch
        g.ext[0], g.ext[1], g.ext[2] = X, Y, Z
    else:
        raise ValueError("grid must be (Y, X, ch) or (Z, Y, X, ch)")
    return g


class Params:
    """sfc_params with the paper's defaults, overridable by keyword."""

    def __init__(self, **kw):
        self.p = sfc_params()
        lib().sfc_params_default(C.byref(self.p))
        self._keep = []
        for k, v in kw.items():
            if k in ("shifts", "ch_weights", "basis", "mean"):
                if v is None:
                    setattr(self.p, k, None)
                    continue
                arr = np.ascontiguousarray(v, np.int32 if k == "shifts" else np.float32)
                self._keep.append(arr)
                setattr(self.p, k, arr.ctypes.data_as(C.c_void_p))
            else:
                setattr(self.p, k, v)

    def __getattr__(self, k):
        return getattr(self.__dict__["p"], k)


class Index:
    """Owner of an sfc_index handle."""

    def __init__(self, handle, params: Params, ndim: int):
        self.h = handle
        self.params = params
        self.ndim = ndim
        N = C.c_int64()
        m = C.c_int32()
        s = C.c_int32()
        _check(lib().sfc_index_info(self.h, C.byref(N), C.byref(m), C.byref(s)), "sfc_index_info")
        self.N, self.m, self.s = N.value, m.value, s.value

    def close(self):
        if self.h:
            lib().sfc_index_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfc_index_build(grid: torch.Tensor, dict_mask: torch.Tensor, **params) -> Index:
    grid = _dev(grid, torch.float32)
    dict_mask = _dev(dict_mask, torch.uint8)
    P = Params(**params)
    g = make_grid(grid)
    h = C.c_void_p()
    _check(lib().sfc_index_build(_ptr(grid), _ptr(dict_mask), C.byref(g), C.byref(P.p), _stream(), C.byref(h)),
           "sfc_index_build")
    return Index(h, P, g.ndim)


def sfc_index_save(ix: Index, path: str) -> None:
    _check(lib().sfc_index_save(ix.h, os.fsencode(path)), "sfc_index_save")


def sfc_index_load(path: str) -> Index:
    h = C.c_void_p()
    _check(lib().sfc_index_load(os.fsencode(path), _stream(), C.byref(h)), "sfc_index_load")
    P = Params()
    g = sfc_grid()
    _check(lib().sfc_index_params(h, C.byref(P.p), C.byref(g)), "sfc_index_params")
    return Index(h, P, g.ndim)


def sfc_query_batch_dict(ix: Index, dict_grid: torch.Tensor, grid: torch.Tensor, cur_mask: torch.Tensor,
                         centres: torch.Tensor, pick: torch.Tensor | None = None, cost: torch.Tensor | None = None):
    """Targets on `grid` (any size, same ndim/channels), dictionary patches from
    `dict_grid` (the grid the index was built from)."""
    dict_grid = _dev(dict_grid, torch.float32)
    grid = _dev(grid, torch.float32)
    cur_mask = _dev(cur_mask, torch.uint8)
    centres = _dev(centres, torch.int32)
    Q = centres.shape[0]
    g = make_grid(grid)
    if pick is None:
        pick = torch.empty(Q, dtype=torch.int64, device=grid.device)
    if cost is None:
        cost = torch.empty(Q, dtype=torch.float32, device=grid.device)
    _check(lib().sfc_query_batch_dict(ix.h, _ptr(dict_grid), _ptr(grid), _ptr(cur_mask), C.byref(g), _ptr(centres),
                                      Q, _ptr(pick), _ptr(cost), _stream()), "sfc_query_batch_dict")
    return pick, cost


def sfc_tune_select(ms, ae, ae_max: float) -> int:
    """The selection rule of sfc_autotune on given measurements (host only)."""
    ms = np.ascontiguousarray(ms, np.float64)
    ae = np.ascontiguousarray(ae, np.float64)
    assert ms.shape == ae.shape and ms.ndim == 1
    return int(lib().sfc_tune_select(len(ms), ms.ctypes.data_as(C.c_void_p), ae.ctypes.data_as(C.c_void_p),
                                     float(ae_max)))


def sfc_autotune(grid: torch.Tensor, mask: torch.Tensor, centres: torch.Tensor, curves=(4, 8), dims=(6, 8, 10),
                 windows=(16, 32, 64, 128), sample: int = 512, reps: int = 3, objective: int = SFC_TUNE_STEP,
                 ae_max: float = 0.01, **base):
    """-> (best params as a dict of the tuned keys, table float64 [n, 5] of
    (C, D, W or k, ms, ae), chosen row)."""
    assert grid.is_cuda and mask.is_cuda
    P = Params(**base)
    g = make_grid(grid)
    cen = _dev(centres, torch.int32)
    lists = [np.ascontiguousarray(v, np.int32) for v in (curves, dims, windows)]
    spec = sfc_tune_spec()
    spec.curves, spec.n_curves = lists[0].ctypes.data_as(C.c_void_p), len(lists[0])
    spec.dims, spec.n_dims = lists[1].ctypes.data_as(C.c_void_p), len(lists[1])
    spec.windows, spec.n_windows = lists[2].ctypes.data_as(C.c_void_p), len(lists[2])
    spec.sample, spec.reps, spec.objective, spec.ae_max = sample, reps, objective, ae_max
    n = len(lists[0]) * len(lists[1]) * len(lists[2])
    table = np.zeros((n, 5), np.float64)
    best = sfc_params()
    chosen = C.c_int32(-1)
    _check(lib().sfc_autotune(_ptr(grid), _ptr(mask), C.byref(g), C.byref(P.p), _ptr(cen), cen.shape[0],
                              C.byref(spec), C.byref(best), table.ctypes.data_as(C.c_void_p), C.byref(chosen),
                              _stream()), "sfc_autotune")
    key = "knn" if P.p.knn > 0 else "window"
    return {"curves": best.curves, "dims": best.dims, key: getattr(best, key)}, table, chosen.value


class Multi:
    """Several indices (same parameters) answered in one launch."""

    def __init__(self, indices, grids, masks):
        n = len(indices)
        self._keep = [(_dev(gr, torch.float32), _dev(mk, torch.uint8)) for gr, mk in zip(grids, masks)]
        self._indices = list(indices)
        hs = (C.c_void_p * n)(*[ix.h for ix in indices])
        gp = (C.c_void_p * n)(*[_ptr(gr) for gr, _ in self._keep])
        mp = (C.c_void_p * n)(*[_ptr(mk) for _, mk in self._keep])
        self.h = C.c_void_p()
        _check(lib().sfc_multi_create(hs, gp, mp, n, _stream(), C.byref(self.h)), "sfc_multi_create")

    def query(self, image: torch.Tensor, centres: torch.Tensor, pick=None, cost=None):
        image = _dev(image, torch.int32)
        centres = _dev(centres, torch.int32)
        Q = centres.shape[0]
        dev = centres.device
        if pick is None:
            pick = torch.empty(Q, dtype=torch.int64, device=dev)
        if cost is None:
            cost = torch.empty(Q, dtype=torch.float32, device=dev)
        _check(lib().sfc_multi_query(self.h, _ptr(image), _ptr(centres), Q, _ptr(pick), _ptr(cost), _stream()),
               "sfc_multi_query")
        return pick, cost

    def close(self):
        if self.h:
            lib().sfc_multi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfc_index_export(ix: Index, proj: bool = False) -> dict:
    C_, D, N, s, m = ix.params.curves, ix.params.dims, ix.N, ix.s, ix.m
    out = dict(dict=np.empty(N, np.int64), subsets=np.empty((C_, m), np.int32), basis=np.empty((C_, s, D), np.float32),
               mean=np.empty((C_, s), np.float32), evals=np.empty((C_, s), np.float64),
               lo=np.empty((C_, D), np.float32), scale=np.empty((C_, D), np.float32),
               skeys=np.empty((C_, N), np.uint64), sids=np.empty((C_, N), np.uint32))
    if proj:
        out["proj"] = np.empty((C_, N, D), np.float32)
        out["keys"] = np.empty((C_, N), np.uint64)
    p = lambda k: out[k].ctypes.data_as(C.c_void_p) if k in out else None  # noqa: E731
    _check(lib().sfc_index_export(ix.h, p("dict"), p("subsets"), p("basis"), p("mean"), p("evals"), p("lo"),
                                  p("scale"), p("proj"), p("keys"), p("skeys"), p("sids")), "sfc_index_export")
    return out


def sfc_query_batch(ix: Index, grid: torch.Tensor, cur_mask: torch.Tensor, centres: torch.Tensor,
                    pick: torch.Tensor | None = None, cost: torch.Tensor | None = None):
    grid = _dev(grid, torch.float32)
    cur_mask = _dev(cur_mask, torch.uint8)
    centres = _dev(centres, torch.int32)
    Q = centres.shape[0]
    if pick is None:
        pick = torch.empty(Q, dtype=torch.int64, device=grid.device)
    if cost is None:
        cost = torch.empty(Q, dtype=torch.float32, device=grid.device)
    _check(lib().sfc_query_batch(ix.h, _ptr(grid), _ptr(cur_mask), _ptr(centres), Q, _ptr(pick), _ptr(cost),
                                 _stream()), "sfc_query_batch")
    return pick, cost


def sfc_query_candidates(ix: Index, grid: torch.Tensor, cur_mask: torch.Tensor, centres: torch.Tensor):
    grid = _dev(grid, torch.float32)
    cur_mask = _dev(cur_mask, torch.uint8)
    centres = _dev(centres, torch.int32)
    Q, C_ = centres.shape[0], ix.params.curves
    W = ix.params.knn if ix.params.knn > 0 else ix.params.window
    dev = grid.device
    qkeys = torch.empty((Q, C_), dtype=torch.int64, device=dev)  # uint64 bits
    pos = torch.empty((Q, C_), dtype=torch.int64, device=dev)
    cand = torch.empty((Q, C_ * W), dtype=torch.int32, device=dev)
    ncand = torch.empty(Q, dtype=torch.int32, device=dev)
    _check(lib().sfc_query_candidates(ix.h, _ptr(grid), _ptr(cur_mask), _ptr(centres), Q, _ptr(qkeys), _ptr(pos),
                                      _ptr(cand), _ptr(ncand), _stream()), "sfc_query_candidates")
    return qkeys, pos, cand, ncand


def fullscan_query_batch(grid: torch.Tensor, dict_mask: torch.Tensor, cur_mask: torch.Tensor,
                         centres: torch.Tensor, K: int, ch_weights=None, pick=None, cost=None,
                         precision: int = SFC_FP32, norm: int = SFC_COST_L2):
    grid = _dev(grid, torch.float32)
    dict_mask = _dev(dict_mask, torch.uint8)
    cur_mask = _dev(cur_mask, torch.uint8)
    centres = _dev(centres, torch.int32)
    Q = centres.shape[0]
    P = Params(K=K, ch_weights=ch_weights, precision=precision, cost=norm)
    g = make_grid(grid)
    if pick is None:
        pick = torch.empty(Q, dtype=torch.int64, device=grid.device)
    if cost is None:
        cost = torch.empty(Q, dtype=torch.float32, device=grid.device)
    _check(lib().fullscan_query_batch(_ptr(grid), _ptr(dict_mask), _ptr(cur_mask), C.byref(g), C.byref(P.p),
                                      _ptr(centres), Q, _ptr(pick), _ptr(cost), _stream()), "fullscan_query_batch")
    return pick, cost


def sfc_tc_prescores(grid: torch.Tensor, dict_mask: torch.Tensor, cur_mask: torch.Tensor, centres: torch.Tensor,
                     K: int, N: int, ch_weights=None):
    """All tensor-core pre-scores (Q x N) and their bounds E_q, for checking."""
    grid = _dev(grid, torch.float32)
    dict_mask = _dev(dict_mask, torch.uint8)
    cur_mask = _dev(cur_mask, torch.uint8)
    centres = _dev(centres, torch.int32)
    Q = centres.shape[0]
    P = Params(K=K, ch_weights=ch_weights, precision=SFC_FP16)
    g = make_grid(grid)
    scores = torch.empty((Q, N), dtype=torch.float32, device=grid.device)
    bound = torch.empty(Q, dtype=torch.float64, device=grid.device)
    n_out = C.c_int64()
    _check(lib().sfc_tc_prescores(_ptr(grid), _ptr(dict_mask), _ptr(cur_mask), C.byref(g), C.byref(P.p),
                                  _ptr(centres), Q, _ptr(scores), _ptr(bound), C.byref(n_out), _stream()),
           "sfc_tc_prescores")
    assert n_out.value == N
    return scores, bound


def fullscan_query_batch_static(grid: torch.Tensor, dict_mask: torch.Tensor, cur_mask: torch.Tensor,
                                centres: torch.Tensor, K: int, ch_weights=None, pick=None, cost=None,
                                norm: int = SFC_COST_L2):
    """As fullscan_query_batch, through the entry point that allocates no device memory."""
    grid = _dev(grid, torch.float32)
    dict_mask = _dev(dict_mask, torch.uint8)
    cur_mask = _dev(cur_mask, torch.uint8)
    centres = _dev(centres, torch.int32)
    Q = centres.shape[0]
    P = Params(K=K, ch_weights=ch_weights, cost=norm)
    g = make_grid(grid)
    if pick is None:
        pick = torch.empty(Q, dtype=torch.int64, device=grid.device)
    if cost is None:
        cost = torch.empty(Q, dtype=torch.float32, device=grid.device)
    _check(lib().fullscan_query_batch_static(_ptr(grid), _ptr(dict_mask), _ptr(cur_mask), C.byref(g),
                                             C.byref(P.p), _ptr(centres), Q, _ptr(pick), _ptr(cost), _stream()),
           "fullscan_query_batch_static")
    return pick, cost


def inpaint_run(grid: torch.Tensor, mask: torch.Tensor, mode: int = SFC_MODE_FULLSCAN, max_steps: int = 0,
                log: bool = True, **params):
    """Runs the fill loop in place on (device) grid and mask.  -> (steps, log int64 [steps, ndim+1])."""
    assert grid.is_cuda and mask.is_cuda and grid.is_contiguous() and mask.is_contiguous()
    assert grid.dtype == torch.float32 and mask.dtype == torch.uint8
    P = Params(**params)
    g = make_grid(grid)
    unknown = int((mask == 0).sum().item())
    cap = unknown if max_steps <= 0 else max_steps
    lg = torch.zeros((max(cap, 1), g.ndim + 1), dtype=torch.int64, device=grid.device) if log else None
    steps = C.c_int64()
    _check(lib().inpaint_run(_ptr(grid), _ptr(mask), C.byref(g), C.byref(P.p), mode, max_steps, _ptr(lg),
                             C.byref(steps), _stream()), "inpaint_run")
    n = steps.value
    return n, (lg[:n] if lg is not None else None)


def sfc_tune_tiles(grid, dict_mask, cur_mask, centres, reps: int = 3, **params):
    """Times the FP32 full scan with each tile shape and keeps the fastest.
    -> (table float64 [shapes, 3] of (queries per tile, entries per thread,
    ms), chosen shape)."""
    grid = _dev(grid, torch.float32)
    dict_mask = _dev(dict_mask, torch.uint8)
    cur_mask = _dev(cur_mask, torch.uint8)
    centres = _dev(centres, torch.int32)
    P = Params(**params)
    g = make_grid(grid)
    table = np.zeros((7, 3), np.float64)
    chosen = C.c_int32(-1)
    _check(lib().sfc_tune_tiles(_ptr(grid), _ptr(dict_mask), _ptr(cur_mask), C.byref(g), C.byref(P.p),
                                _ptr(centres), centres.shape[0], reps, table.ctypes.data_as(C.c_void_p),
                                C.byref(chosen), _stream()), "sfc_tune_tiles")
    return table, chosen.value


def sfc_tile_shape(shape: int = -1) -> int:
    """Sets the FP32 full scan's tile shape (0..6; other values only read it)."""
    return int(lib().sfc_tile_shape(int(shape)))


def inpaint_run_multi(grids, masks, max_steps: int = 0, log: bool = True, **params):
    """The fill loops of several images at once (SFC mode), in place on the
    (device) grids and masks.  -> (steps per image, logs: list of int64
    [steps, ndim+1] or None)."""
    n = len(grids)
    assert n == len(masks) and n >= 1
    for g_, m_ in zip(grids, masks):
        assert g_.is_cuda and m_.is_cuda and g_.is_contiguous() and m_.is_contiguous()
        assert g_.dtype == torch.float32 and m_.dtype == torch.uint8
    P = Params(**params)
    gs = (sfc_grid * n)(*[make_grid(g_) for g_ in grids])
    logs = []
    for g_, m_ in zip(grids, masks):
        unknown = int((m_ == 0).sum().item())
        cap = unknown if max_steps <= 0 else max_steps
        nd = gs[0].ndim
        logs.append(torch.zeros((max(cap, 1), nd + 1), dtype=torch.int64, device=g_.device) if log else None)
    gp = (C.c_void_p * n)(*[_ptr(g_) for g_ in grids])
    mp = (C.c_void_p * n)(*[_ptr(m_) for m_ in masks])
    lp = (C.c_void_p * n)(*[_ptr(l_) for l_ in logs]) if log else None
    steps = np.zeros(n, np.int64)
    _check(lib().inpaint_run_multi(gp, mp, gs, n, C.byref(P.p), max_steps, lp, steps.ctypes.data_as(C.c_void_p),
                                   _stream()), "inpaint_run_multi")
    return steps.tolist(), ([l_[:k] for l_, k in zip(logs, steps)] if log else None)


def sfc_launch_count() -> int:
    return int(lib().sfc_launch_count())


def sfc_trace(on: bool) -> None:
    _check(lib().sfc_trace(1 if on else 0), "sfc_trace")


def sfc_trace_read() -> dict:
    ms = np.zeros(len(TRACE_PHASES), np.float64)
    builds = np.zeros(1, np.int64)
    fl = np.zeros(1, np.float64)
    _check(lib().sfc_trace_read(ms.ctypes.data_as(C.c_void_p), builds.ctypes.data_as(C.c_void_p),
                                fl.ctypes.data_as(C.c_void_p)), "sfc_trace_read")
    f64 = np.zeros(1, np.float64)
    f32 = np.zeros(1, np.float64)
    _check(lib().sfc_trace_eig_read(f64.ctypes.data_as(C.c_void_p), f32.ctypes.data_as(C.c_void_p)),
           "sfc_trace_eig_read")
    return dict(ms=dict(zip(TRACE_PHASES, ms.tolist())), builds=int(builds[0]), eig_flops=float(fl[0]),
                eig_flops32=float(f32[0]))


TRACE_TC_PHASES = ("operands", "gemm", "exact")


def sfc_trace_tc_read() -> dict:
    ms = np.zeros(len(TRACE_TC_PHASES), np.float64)
    calls = np.zeros(1, np.int64)
    fl = np.zeros(1, np.float64)
    _check(lib().sfc_trace_tc_read(ms.ctypes.data_as(C.c_void_p), calls.ctypes.data_as(C.c_void_p),
                                   fl.ctypes.data_as(C.c_void_p)), "sfc_trace_tc_read")
    return dict(ms=dict(zip(TRACE_TC_PHASES, ms.tolist())), calls=int(calls[0]), gemm_flops=float(fl[0]))


def sfc_status() -> int:
    return lib().sfc_status(_stream())


def sfc_trace_proj_read() -> dict:
    """Summed time, builds counted and algorithmic work of the traced projection launches."""
    ms, fl, by = C.c_double(), C.c_double(), C.c_double()
    calls = C.c_int64()
    _check(lib().sfc_trace_proj_read(C.byref(ms), C.byref(calls), C.byref(fl), C.byref(by)), "sfc_trace_proj_read")
    return {"ms": ms.value, "calls": calls.value, "flops": fl.value, "bytes": by.value}


def sfc_debug_fail_alloc(n: int) -> None:
    """Failure injection (tests): the n-th library allocation from now on fails (0: off)."""
    _check(lib().sfc_debug_fail_alloc(int(n)), "sfc_debug_fail_alloc")


def sfc_debug_alloc_count() -> int:
    return int(lib().sfc_debug_alloc_count())


def sfc_debug_pool_used() -> int:
    v = C.c_uint64()
    _check(lib().sfc_debug_pool_used(C.byref(v)), "sfc_debug_pool_used")
    return int(v.value)


def sfc_debug_lookback(spin_limit: int = 0, stall: bool = False) -> None:
    """Failure injection (tests): the radix sort's look-back poll limit and stall switch."""
    _check(lib().sfc_debug_lookback(int(spin_limit), 1 if stall else 0), "sfc_debug_lookback")


def sfc_debug_sort(force_lsd: bool = False, bucket_cap: int = 0) -> None:
    """Builds sort with the LSD radix sort (force_lsd), or the sample sort with
    a lowered bucket capacity (its LSD fallback); (False, 0) resets."""
    _check(lib().sfc_debug_sort(1 if force_lsd else 0, int(bucket_cap)), "sfc_debug_sort")