"""CPU oracle for the SFC-indexed exemplar-inpainting patch search.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  It shares no code with the CUDA
library.  ``sfc_oracle.cpp`` holds the arithmetic (plain single-threaded C++,
``-O2 -ffp-contract=off``); this module compiles it with g++ and marshals
numpy arrays through ctypes.  Each helper names the paper passage its C
function follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfc_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

P = C.c_void_p
I64 = C.c_int64
I32 = C.c_int


def build(force: bool = False) -> str:
    """Compile the oracle (g++, no fast-math, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            sig = {
                "or_dict_extract": (I64, [P, I32, P, I32, P, I64]),
                "or_cost64": (C.c_double, [P, P, I32, P, I32, I32, I64, I64, P, I32]),
                "or_fullscan": (None, [P, P, I32, P, I32, I32, P, I64, P, I64, P, P, P, I32]),
                "or_subsets": (I32, [I32, I32, C.c_double, I32, P, P]),
                "or_jacobi": (I32, [P, I32, P, P, I32]),
                "or_pca": (I32, [P, I32, P, I32, I32, P, I64, P, I32, I64, I32, P, P, P, P]),
                "or_project_one": (None, [P, P, I32, P, I32, I32, I64, P, I32, P, P, I32, P]),
                "or_project": (None, [P, I32, P, I32, I32, P, I64, P, I32, P, P, I32, P]),
                "or_quant_params": (None, [P, I64, I32, I32, P, P]),
                "or_quantise": (None, [P, I64, I32, I32, P, P, P]),
                "or_morton": (C.c_uint64, [P, I32, I32]),
                "or_key_bits": (I32, [I32, I32, P]),
                "or_keys": (None, [P, I64, I32, I32, P, P]),
                "or_keys_curve": (None, [P, I64, I32, I32, P, I32, P]),
                "or_hilbert": (C.c_uint64, [P, I32, I32]),
                "or_query_curve": (None, [P, P, I32, P, I32, I32, I32, I32, I32, I32, I32, P, P, I32, P, P, P, P,
                                          P, I32, P, P, P, I64, I64, P, P, P, P, P, P, I32]),
                "or_zless": (I32, [P, P, I32]),
                "or_sort": (None, [P, I64, P, P]),
                "or_lower_bound": (I64, [P, I64, C.c_uint64]),
                "or_query": (None, [P, P, I32, P, I32, I32, I32, I32, I32, I32, I32, P, P, I32, P, P, P, P, P,
                                    P, P, P, I64, I64, P, P, P, P, P, P]),
                "or_knn_bruteforce": (None, [P, I64, I32, P, I32, P, P]),
                "or_cost64_2": (C.c_double, [P, P, I32, P, P, P, I32, I32, I64, I64, P, I32]),
                "or_query_dict": (None, [P, P, P, P, P, I32, I32, I32, I32, I32, I32, I32, I32, P, P, I32, P, P, P,
                                         P, P, I32, P, P, P, I64, I64, P, P, P, P, I32]),
                "or_query_knn": (None, [P, P, I32, P, I32, I32, I32, I32, I32, I32, I32, P, P, I32, P, P, P, P, P,
                                        P, I64, I64, P, P, P, P, I32]),
                "or_priority": (I32, [P, P, P, I32, P, I32, I32, I64, I32, P]),
                "or_inpaint": (I64, [P, P, I32, P, I32, I32, I32, I32, P, P, I64, I32, I32, I32, I32, I32, P,
                                     I32, P, P, P, P, P, P, P, I64, P, I32, I32, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def geometry(grid: np.ndarray):
    """(ndim, ext[X, Y, Z], ch) of a grid laid out (Y, X, ch) or (Z, Y, X, ch)."""
    if grid.ndim == 3:
        Y, X, ch = grid.shape
        return 2, np.array([X, Y, 1], np.int64), ch
    Z, Y, X, ch = grid.shape
    return 3, np.array([X, Y, Z], np.int64), ch


def centres_to_lin(centres: np.ndarray, ext) -> np.ndarray:
    centres = np.asarray(centres, np.int64)
    lin = centres[:, 0].copy()
    mul = int(ext[0])
    for a in range(1, centres.shape[1]):
        lin += centres[:, a] * mul
        mul *= int(ext[a])
    return lin


def lin_to_centres(lin: np.ndarray, ext, ndim: int) -> np.ndarray:
    lin = np.asarray(lin, np.int64)
    out = np.empty((len(lin), ndim), np.int64)
    rem = lin.copy()
    for a in range(ndim):
        out[:, a] = rem % int(ext[a])
        rem //= int(ext[a])
    return out


# ----------------------------------------------------------------------------
def dict_extract(mask: np.ndarray, K: int) -> np.ndarray:
    """Dictionary of fully known patches (Sec. I), centre linear indices in raster order."""
    ndim = mask.ndim
    ext = np.array(list(mask.shape[::-1]) + [1] * (3 - ndim), np.int64)
    m = _c(mask, np.uint8)
    n = lib().or_dict_extract(_p(m), ndim, _p(ext), K, None, 0)
    out = np.empty(n, np.int64)
    lib().or_dict_extract(_p(m), ndim, _p(ext), K, _p(out), n)
    return out


def cost64(grid, cur_mask, K, target_lin, source_lin, weights=None, norm=0) -> float:
    ndim, ext, ch = geometry(grid)
    w = None if weights is None else _c(weights, np.float32)
    return lib().or_cost64(_p(_c(grid, np.float32)), _p(_c(cur_mask, np.uint8)), ndim, _p(ext), ch, K,
                           int(target_lin), int(source_lin), _p(w), int(norm))


def fullscan(grid, cur_mask, K, dict_lin, targets_lin, weights=None, norm=0):
    """Full scan + global argmin, ties to the lowest id (Sec. I).  -> (pick int64[Q], cost float64[Q])."""
    ndim, ext, ch = geometry(grid)
    g = _c(grid, np.float32)
    m = _c(cur_mask, np.uint8)
    d = _c(dict_lin, np.int64)
    t = _c(targets_lin, np.int64)
    w = None if weights is None else _c(weights, np.float32)
    pick = np.empty(len(t), np.int64)
    cost = np.empty(len(t), np.float64)
    lib().or_fullscan(_p(g), _p(m), ndim, _p(ext), ch, K, _p(d), len(d), _p(t), len(t), _p(w), _p(pick), _p(cost),
                      norm)
    return pick, cost


def subsets(ndim: int, K: int, frac: float, C_: int) -> np.ndarray:
    """Pixel subsets of the indices (Fig. 2) -> int32 [C, m] patch pixel indices."""
    P_ = K ** ndim
    out = np.empty(C_ * P_, np.int32)
    m = np.zeros(1, np.int32)
    rc = lib().or_subsets(ndim, K, float(frac), C_, _p(out), _p(m))
    if rc != 0:
        raise ValueError("too many indices for the available anchors")
    return out[: C_ * int(m[0])].reshape(C_, int(m[0])).copy()


def jacobi(A: np.ndarray, max_sweeps: int = 100):
    """Cyclic Jacobi eigen-decomposition (textbook) -> (evals, V, sweeps); columns of V are eigenvectors."""
    n = A.shape[0]
    a = _c(A, np.float64).copy()
    ev = np.empty(n, np.float64)
    V = np.empty((n, n), np.float64)
    sw = lib().or_jacobi(_p(a), n, _p(ev), _p(V), max_sweeps)
    return ev, V, sw


def pca(grid, K, dict_lin, subset_row, sample, D):
    """PCA of one index (Sec. II.A) -> (basis f32 [s, D], mean f32 [s], evals f64 [s], cov f64 [s, s])."""
    ndim, ext, ch = geometry(grid)
    m = len(subset_row)
    s = m * ch
    basis = np.empty((s, D), np.float32)
    mean = np.empty(s, np.float32)
    ev = np.empty(s, np.float64)
    cov = np.empty((s, s), np.float64)
    lib().or_pca(_p(_c(grid, np.float32)), ndim, _p(ext), ch, K, _p(_c(dict_lin, np.int64)), len(dict_lin),
                 _p(_c(subset_row, np.int32)), m, int(sample), D, _p(basis), _p(mean), _p(ev), _p(cov))
    return basis, mean, ev, cov


def project(grid, K, dict_lin, subset_row, basis, mean, D):
    ndim, ext, ch = geometry(grid)
    y = np.empty((len(dict_lin), D), np.float32)
    lib().or_project(_p(_c(grid, np.float32)), ndim, _p(ext), ch, K, _p(_c(dict_lin, np.int64)), len(dict_lin),
                     _p(_c(subset_row, np.int32)), len(subset_row), _p(_c(basis, np.float32)),
                     _p(_c(mean, np.float32)), D, _p(y))
    return y


def project_query(grid, cur_mask, K, centre_lin, subset_row, basis, mean, D):
    ndim, ext, ch = geometry(grid)
    y = np.empty(D, np.float32)
    lib().or_project_one(_p(_c(grid, np.float32)), _p(_c(cur_mask, np.uint8)), ndim, _p(ext), ch, K,
                         int(centre_lin), _p(_c(subset_row, np.int32)), len(subset_row), _p(_c(basis, np.float32)),
                         _p(_c(mean, np.float32)), D, _p(y))
    return y


def quant_params(y, bits):
    N, D = y.shape
    lo = np.empty(D, np.float32)
    sc = np.empty(D, np.float32)
    lib().or_quant_params(_p(_c(y, np.float32)), N, D, bits, _p(lo), _p(sc))
    return lo, sc


def quantise(y, bits, lo, scale):
    N, D = y.shape
    q = np.empty((N, D), np.uint32)
    lib().or_quantise(_p(_c(y, np.float32)), N, D, bits, _p(_c(lo, np.float32)), _p(_c(scale, np.float32)), _p(q))
    return q


def morton(q, bp) -> int:
    q = _c(q, np.uint32)
    return int(lib().or_morton(_p(q), len(q), bp))


def key_bits(D, bits, shift=None) -> int:
    sh = None if shift is None else _c(shift, np.int32)
    return int(lib().or_key_bits(D, bits, _p(sh)))


def keys(q, bits, shift=None, curve=0):
    """Curve keys of quantised points: curve 0 = Morton (Sec. II.C), 1 = Hilbert."""
    N, D = q.shape
    out = np.empty(N, np.uint64)
    sh = None if shift is None else _c(shift, np.int32)
    lib().or_keys_curve(_p(_c(q, np.uint32)), N, D, bits, _p(sh), curve, _p(out))
    return out


def hilbert(q, bp) -> int:
    q = _c(q, np.uint32)
    return int(lib().or_hilbert(_p(q), len(q), bp))


def zless(a, b) -> bool:
    a = _c(a, np.uint32)
    b = _c(b, np.uint32)
    return bool(lib().or_zless(_p(a), _p(b), len(a)))


def sort(k):
    N = len(k)
    sk = np.empty(N, np.uint64)
    si = np.empty(N, np.uint32)
    lib().or_sort(_p(_c(k, np.uint64)), N, _p(sk), _p(si))
    return sk, si


def lower_bound(skeys, key) -> int:
    return int(lib().or_lower_bound(_p(_c(skeys, np.uint64)), len(skeys), C.c_uint64(int(key))))


def knn_bruteforce(qcoords, query, k):
    N, D = qcoords.shape
    kk = min(k, N)
    out = np.empty(kk, np.int64)
    dist = np.empty(kk, np.int64)
    lib().or_knn_bruteforce(_p(_c(qcoords, np.uint32)), N, D, _p(_c(query, np.uint32)), k, _p(out), _p(dist))
    return out, dist


# ----------------------------------------------------------------------------
# Index (Sec. II.A-C) and query (Fig. 1) built from the functions above
# ----------------------------------------------------------------------------
def build_index(grid, mask, K, C_, D, bits, frac=0.6, sample=1 << 20, shifts=None, basis=None, mean=None, curve=0):
    """All arrays of the multi-index.  ``basis``/``mean`` ([C, s, D] / [C, s]) may
    be given to build from a common basis (e.g. one exported from the GPU);
    otherwise the oracle's own PCA is used."""
    ndim, ext, ch = geometry(grid)
    dct = dict_extract(mask, K)
    sub = subsets(ndim, K, frac, C_)
    m = sub.shape[1]
    s = m * ch
    N = len(dct)
    B = np.empty((C_, s, D), np.float32)
    MU = np.empty((C_, s), np.float32)
    EV = np.empty((C_, s), np.float64)
    Y = np.empty((C_, N, D), np.float32)
    LO = np.empty((C_, D), np.float32)
    SC = np.empty((C_, D), np.float32)
    Q = np.empty((C_, N, D), np.uint32)
    KEYS = np.empty((C_, N), np.uint64)
    SK = np.empty((C_, N), np.uint64)
    SI = np.empty((C_, N), np.uint32)
    sh = None if shifts is None else np.ascontiguousarray(shifts, np.int32).reshape(C_, D)
    for cv in range(C_):
        if basis is None:
            B[cv], MU[cv], EV[cv], _ = pca(grid, K, dct, sub[cv], sample, D)
        else:
            B[cv] = basis[cv]
            MU[cv] = mean[cv]
            EV[cv] = np.nan
        Y[cv] = project(grid, K, dct, sub[cv], B[cv], MU[cv], D)
        LO[cv], SC[cv] = quant_params(Y[cv], bits)
        Q[cv] = quantise(Y[cv], bits, LO[cv], SC[cv])
        KEYS[cv] = keys(Q[cv], bits, None if sh is None else sh[cv], curve)
        SK[cv], SI[cv] = sort(KEYS[cv])
    return dict(ndim=ndim, ext=ext, ch=ch, K=K, C=C_, D=D, bits=bits, dict=dct, N=N, subset=sub, m=m, basis=B,
                mean=MU, evals=EV, proj=Y, lo=LO, scale=SC, q=Q, keys=KEYS, skeys=SK, sids=SI, shifts=sh,
                curve=curve)


def query(ix, grid, cur_mask, target_lin, W, select=0, weights=None, norm=0):
    """One SFC query (Fig. 1(b)-(d)) -> dict(pick, cost, cand, qkeys, pos)."""
    ndim, ext, ch = geometry(grid)
    C_, D = ix["C"], ix["D"]
    qk = np.zeros(C_, np.uint64)
    pos = np.zeros(C_, np.int64)
    cand = np.empty(C_ * max(W, 1), np.int64)
    nc = np.zeros(1, np.int64)
    pick = np.zeros(1, np.int64)
    cost = np.zeros(1, np.float64)
    w = None if weights is None else _c(weights, np.float32)
    lib().or_query_curve(_p(_c(grid, np.float32)), _p(_c(cur_mask, np.uint8)), ndim, _p(ext), ch, ix["K"], C_, D,
                         ix["bits"], W, select, _p(w), _p(ix["subset"]), ix["m"], _p(ix["basis"]), _p(ix["mean"]),
                         _p(ix["lo"]), _p(ix["scale"]), _p(ix["shifts"]), int(ix.get("curve", 0)), _p(ix["skeys"]),
                         _p(ix["sids"]), _p(ix["dict"]), ix["N"], int(target_lin), _p(qk), _p(pos), _p(cand),
                         _p(nc), _p(pick), _p(cost), int(norm))
    return dict(pick=int(pick[0]), cost=float(cost[0]), cand=cand[: int(nc[0])].copy(), qkeys=qk, pos=pos)


def cost64_2(tgrid, tmask, dgrid, K, target_lin, source_lin, weights=None, norm=0) -> float:
    """cost64 with the target patch from tgrid/tmask and the source patch from dgrid."""
    ndim, text, ch = geometry(tgrid)
    _, dext, dch = geometry(dgrid)
    assert dch == ch
    w = None if weights is None else _c(weights, np.float32)
    return lib().or_cost64_2(_p(_c(tgrid, np.float32)), _p(_c(tmask, np.uint8)), ndim, _p(text),
                             _p(_c(dgrid, np.float32)), _p(dext), ch, K, int(target_lin), int(source_lin), _p(w),
                             int(norm))


def query_dict(ix, dict_grid, grid, cur_mask, target_lin, W, select=0, weights=None, norm=0):
    """SFC query of a target in (grid, cur_mask) against an index whose dictionary
    patches are in dict_grid -> dict(pick, cost, cand)."""
    ndim, text, ch = geometry(grid)
    _, dext, _ = geometry(dict_grid)
    C_, D = ix["C"], ix["D"]
    cand = np.empty(C_ * max(W, 1), np.int64)
    nc = np.zeros(1, np.int64)
    pick = np.zeros(1, np.int64)
    cost = np.zeros(1, np.float64)
    w = None if weights is None else _c(weights, np.float32)
    lib().or_query_dict(_p(_c(dict_grid, np.float32)), _p(dext), _p(_c(grid, np.float32)),
                        _p(_c(cur_mask, np.uint8)), _p(text), ndim, ch, ix["K"], C_, D, ix["bits"], W, select,
                        _p(w), _p(_c(ix["subset"], np.int32)), ix["m"], _p(_c(ix["basis"], np.float32)),
                        _p(_c(ix["mean"], np.float32)), _p(_c(ix["lo"], np.float32)), _p(_c(ix["scale"], np.float32)),
                        _p(ix["shifts"]), int(ix.get("curve", 0)), _p(ix["skeys"]), _p(ix["sids"]),
                        _p(_c(ix["dict"], np.int64)), ix["N"], int(target_lin), _p(cand), _p(nc), _p(pick), _p(cost),
                        int(norm))
    return dict(pick=int(pick[0]), cost=float(cost[0]), cand=cand[: int(nc[0])].copy())


def query_knn(ix, grid, cur_mask, target_lin, k, select=0, weights=None, norm=0):
    """One SFC query with exact k-NN lists (Sec. II.D) -> dict(pick, cost, cand).
    ``ix`` needs "q": [C, N, D] unshifted quantised coordinates."""
    ndim, ext, ch = geometry(grid)
    C_, D = ix["C"], ix["D"]
    cand = np.empty(C_ * max(k, 1), np.int64)
    nc = np.zeros(1, np.int64)
    pick = np.zeros(1, np.int64)
    cost = np.zeros(1, np.float64)
    w = None if weights is None else _c(weights, np.float32)
    lib().or_query_knn(_p(_c(grid, np.float32)), _p(_c(cur_mask, np.uint8)), ndim, _p(ext), ch, ix["K"], C_, D,
                       ix["bits"], k, select, _p(w), _p(_c(ix["subset"], np.int32)), ix["m"],
                       _p(_c(ix["basis"], np.float32)), _p(_c(ix["mean"], np.float32)), _p(_c(ix["lo"], np.float32)),
                       _p(_c(ix["scale"], np.float32)), _p(_c(ix["q"], np.uint32)), _p(_c(ix["dict"], np.int64)),
                       ix["N"], int(target_lin), _p(cand), _p(nc), _p(pick), _p(cost), int(norm))
    return dict(pick=int(pick[0]), cost=float(cost[0]), cand=cand[: int(nc[0])].copy())


def priority(grid, mask, K, centre_xy, prio=1, conf=None):
    """Fill-order terms of one centre (the Criminisi priority the paper defers
    to, Sec. I) -> dict C, gx, gy, nx, ny, D, P (all float32 values)."""
    ndim, ext, ch = geometry(grid)
    terms = np.zeros(7, np.float32)
    lin = int(centres_to_lin(np.array([centre_xy]), ext)[0])
    cf = None if conf is None else _c(conf, np.float32)
    rc = lib().or_priority(_p(_c(grid, np.float32)), _p(_c(mask, np.uint8)), _p(cf), ndim, _p(ext), ch, K, lin,
                           int(prio), _p(terms))
    if rc != 0:
        raise ValueError(f"or_priority: {rc}")
    return dict(zip(("C", "gx", "gy", "nx", "ny", "D", "P"), (float(v) for v in terms)))


def inpaint(grid, mask, K, mode=0, prio=0, ix=None, W=64, select=0, weights=None, max_steps=0, norm=0, knn=0):
    """Fill loop (Sec. I, Fig. 1(a)); works on copies.  mode 0 = full scan,
    1 = SFC (needs ``ix``): windows of W, or with knn > 0 the exact k-NN lists
    of Sec. II.D.  -> (grid, mask, log int64 [steps, ndim+1], steps)."""
    ndim, ext, ch = geometry(grid)
    g = np.array(grid, np.float32, copy=True)
    m = np.array(mask, np.uint8, copy=True)
    dct = dict_extract(mask, K) if ix is None else ix["dict"]
    w = None if weights is None else _c(weights, np.float32)
    unknown = int((m == 0).sum())
    cap = max(unknown, 1) if max_steps <= 0 else max_steps
    log = np.zeros((cap, ndim + 1), np.int64)
    if ix is None:
        args = [0, 0, 0, 0, 0, None, 0, None, None, None, None, None, None, None]
    else:
        args = [ix["C"], ix["D"], ix["bits"], W, select, _p(ix["subset"]), ix["m"], _p(ix["basis"]),
                _p(ix["mean"]), _p(ix["lo"]), _p(ix["scale"]), _p(ix["shifts"]), _p(ix["skeys"]), _p(ix["sids"])]
    steps = lib().or_inpaint(_p(g), _p(m), ndim, _p(ext), ch, K, mode, prio, _p(w), _p(_c(dct, np.int64)), len(dct),
                             *args, int(max_steps), _p(log), int(norm), int(knn),
                             _p(_c(ix["q"], np.uint32)) if (ix is not None and knn > 0) else None)
    if steps < 0:
        raise ValueError(f"oracle inpaint failed ({steps})")
    return g, m, log[:steps].copy(), int(steps)
