"""The C-ABI library loads without a GPU, exports every symbol its header
declares, and rejects invalid arguments before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1712_06326_gb300 import sfc

    return sfc.lib()


def header_functions():
    names = []
    for path in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not path.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", path)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", txt, re.M):
            names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = header_functions()
    for must in ["sfc_index_build", "sfc_query_batch", "fullscan_query_batch", "inpaint_run"]:
        assert must in names


def test_every_declared_symbol_is_exported(L):
    for name in header_functions():
        assert hasattr(L, name), f"{name} declared in include/ but not exported"


def test_params_default_is_the_papers(L):
    from paper_1712_06326_gb300 import sfc

    p = sfc.sfc_params()
    L.sfc_params_default(C.byref(p))
    assert (p.K, p.curves, p.dims, p.window) == (9, 8, 10, 80)
    assert abs(p.subset_frac - 0.6) < 1e-7


def test_invalid_arguments_rejected_on_host(L):
    from paper_1712_06326_gb300 import sfc

    g = sfc.sfc_grid()
    p = sfc.sfc_params()
    L.sfc_params_default(C.byref(p))
    assert L.sfc_index_build(None, None, C.byref(g), C.byref(p), None, None) == sfc.SFC_EINVAL
    assert L.sfc_query_batch(None, None, None, None, 4, None, None, None) == sfc.SFC_EINVAL
    assert L.sfc_query_batch(None, None, None, None, -1, None, None, None) == sfc.SFC_EINVAL
    assert L.fullscan_query_batch(None, None, None, C.byref(g), C.byref(p), None, 3, None, None, None) == sfc.SFC_EINVAL
    steps = C.c_int64()
    assert L.inpaint_run(None, None, C.byref(g), C.byref(p), 0, 0, None, C.byref(steps), None) == sfc.SFC_EINVAL
    assert L.sfc_index_destroy(None) == 0
    assert len(L.sfc_last_error()) > 0
    # the many-image fill loop and the tile-shape tuner check their arguments first
    st = (C.c_int64 * 2)()
    assert L.inpaint_run_multi(None, None, None, 0, C.byref(p), 0, None, st, None) == sfc.SFC_EINVAL
    assert L.inpaint_run_multi(None, None, C.byref(g), 2, C.byref(p), 0, None, st, None) == sfc.SFC_EINVAL
    table = (C.c_double * 21)()
    assert L.sfc_tune_tiles(None, None, None, C.byref(g), C.byref(p), None, 4, 2, table, None, None) == sfc.SFC_EINVAL
    # reading the full scan's tile shape touches no device
    assert L.sfc_tile_shape(-1) == 0


def test_library_has_no_cpu_fallback_symbols(L):
    # the product library never links the oracle
    import subprocess

    out = subprocess.run(["nm", "-D", sfc_lib_path()], capture_output=True, text=True).stdout
    assert "or_fullscan" not in out and "or_query" not in out


def sfc_lib_path():
    from paper_1712_06326_gb300 import sfc

    return sfc.LIB_PATH
