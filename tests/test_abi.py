"""Host-side checks of the C ABI: the library builds for sm_103a, loads
without a GPU and exports every function include/gj.h declares."""
import ctypes

from paper_2206_10435_gb300 import build, gj


def test_header_declares_the_boundary_calls():
    names = gj.header_functions()
    for required in ["gj_create", "gj_destroy", "gj_load_relation", "gj_build_factors",
                     "gj_query_create", "gj_summarize", "gj_summary_groups", "gj_level",
                     "gj_desummarize", "gj_query_destroy", "gj_status_str"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    build.build()
    L = ctypes.CDLL(build.LIB)
    missing = [n for n in gj.header_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    L = gj.lib()
    assert L.gj_version() >= 1
    for s in range(9):
        assert L.gj_status_str(s)
    assert L.gj_status_str(gj.GJ_ERR_OVERFLOW) == b"join size reaches 2^64 - 1"


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        return
    h = ctypes.c_void_p()
    st = gj.lib().gj_create(ctypes.byref(h), 0, None)
    assert st == gj.GJ_ERR_CUDA and not h.value


def test_binding_constants_match_the_header():
    # every GJ_* value the Python binding mirrors (status codes, relation
    # flags, options) is the one include/gj.h defines
    import re
    text = open(gj.HEADER).read()
    defs = {m.group(1): int(m.group(2)) for m in
            re.finditer(r"^\s*#define\s+(GJ_[A-Z0-9_]+)\s+(\d+)u?\s*(?:/\*.*)?$", text, re.M)}
    defs.update({m.group(1): int(m.group(2)) for m in
                 re.finditer(r"^\s*(GJ_[A-Z0-9_]+)\s*=\s*(\d+)\s*,?", text, re.M)})
    mirrored = {n: getattr(gj, n) for n in dir(gj) if n.startswith("GJ_") and isinstance(getattr(gj, n), int)}
    assert {"GJ_OK", "GJ_ERR_CAPACITY", "GJ_REL_HOST", "GJ_OPT_TRIANGLE_INTERSECT"} <= set(mirrored)
    for n, v in mirrored.items():
        assert n in defs, n
        assert defs[n] == v, (n, defs[n], v)


def test_every_entry_point_rejects_null_handles():
    # the boundary's error behaviour: NULL handles and pointers give
    # GJ_ERR_INVALID (destroy calls are no-ops), never a crash; no GPU needed
    L = ctypes.CDLL(build.LIB)
    void_fns = {"gj_destroy", "gj_query_destroy", "gj_batch_destroy", "gj_server_destroy"}
    for name in gj.header_functions():
        if name in ("gj_status_str", "gj_version", "gj_last_error"):
            continue
        f = getattr(L, name)
        f.restype = None if name in void_fns else ctypes.c_int
        r = f(*([None] * 12))
        if name not in void_fns:
            assert r == gj.GJ_ERR_INVALID, (name, r)
