"""gj_factor_build_noalloc builds the frequency table of one relation with
all of its scratch in the library's fixed device array, for callers that
cannot allocate device memory (an engine that owns every byte of device
memory through its own pool, or a latency-critical path where cudaMalloc
would synchronise the device).  Its output must equal the allocating entry
point's (gj_build_factors + gj_factor_export) exactly, call after call, even
though every call reuses the same scratch.

This file is named to be collected last: the entry point keeps state in a
device array shared by every call, so the rest of the suite runs first."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(L, gj, cols, order, n_rows):
    n = max(n_rows, 1)
    perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    gstart = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
    gkey = torch.full((len(cols) * n,), -1, dtype=torch.int32, device="cuda")
    G = ctypes.c_int64(-1)
    kp = (ctypes.c_void_p * len(cols))(*[t.data_ptr() for t in cols])
    co = (ctypes.c_int32 * len(order))(*order)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.gj_factor_build_noalloc(0, stream, n_rows, len(cols), kp, co,
                                   ctypes.c_void_p(perm.data_ptr()),
                                   ctypes.c_void_p(gstart.data_ptr()),
                                   ctypes.c_void_p(gkey.data_ptr()), ctypes.byref(G))
    return st, G.value, perm[:n_rows], gstart, gkey


def test_noalloc_factor_equals_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_10435_gb300 import gj
    L = gj.lib()
    rng = np.random.default_rng(11)
    n_max = 1 << 18
    # two relations of different sizes and widths, built alternately so that
    # every call starts from the previous call's leftovers in the scratch
    rels = []
    for n, spec in ((n_max, [(-50, 3000), (0, 1 << 30), (0, 40)]), (100_003, [(0, 7), (-9, 9)])):
        cols = [torch.from_numpy(rng.integers(lo, hi, n, dtype=np.int32)).cuda() for lo, hi in spec]
        rels.append((n, cols))
    ctx = gj.Context(0)
    ids = [ctx.load_relation(cols, list(range(len(cols)))) for n, cols in rels]
    calls = [(0, [0, 1, 2]), (1, [1, 0]), (0, [2, 0, 1]), (1, [0, 1])]
    for which, order in calls:
        n, cols = rels[which]
        ref_perm, ref_gstart, ref_gkey = ctx.factor_export(ids[which], n, len(cols), order)
        for _ in range(2):   # two calls in a row on the same input
            st, G, perm, gstart, gkey = _noalloc(L, gj, cols, order, n)
            torch.cuda.synchronize()
            assert st == gj.GJ_OK, L.gj_status_str(st)
            assert G == ref_gstart.numel() - 1
            assert torch.equal(perm, ref_perm)
            assert torch.equal(gstart[:G + 1], ref_gstart)
            assert torch.equal(gkey[:len(cols) * G].view(len(cols), G), ref_gkey)
    # an empty relation (no groups, gstart = [0]) and a one-row relation (one
    # group) skip the sort; both still match the allocating path
    for n_small in (0, 1):
        small = [torch.from_numpy(rng.integers(-5, 5, n_small, dtype=np.int32)).cuda() for _ in range(2)]
        sid = ctx.load_relation(small, [0, 1])
        ref_perm, ref_gstart, ref_gkey = ctx.factor_export(sid, n_small, 2, [1, 0])
        for _ in range(2):
            st, G, perm, gstart, gkey = _noalloc(L, gj, small, [1, 0], n_small)
            torch.cuda.synchronize()
            assert st == gj.GJ_OK, L.gj_status_str(st)
            assert G == n_small == ref_gstart.numel() - 1
            assert torch.equal(perm, ref_perm[:n_small])
            assert torch.equal(gstart[:G + 1], ref_gstart)
            assert torch.equal(gkey[:2 * G].view(2, G), ref_gkey.view(2, G))
        ctx.release_relation(sid)
    # sizes beyond the fixed scratch are refused before any work
    n, cols = rels[0]
    st, G, *_ = _noalloc(L, gj, cols, [0, 1, 2], n_max + 1)
    assert st == gj.GJ_ERR_INVALID and G == 0
    for i in ids:
        ctx.release_relation(i)
    ctx.close()
