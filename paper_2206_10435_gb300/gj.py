"""Python binding of libgj.so (include/gj.h): argument marshalling only.

Every step of the join runs in the library's CUDA kernels; this module only
turns torch tensors into device pointers and C structs.  There is no CPU
fallback: if the compiled library is missing the import of ``lib()`` fails.

The entry points keep the C names (``gj_create``, ``gj_load_relation``,
``gj_build_factors``, ``gj_query_create``, ``gj_summarize``,
``gj_summary_groups``, ``gj_level``, ``gj_desummarize`` ...).  ``Context`` and
``Query`` wrap them for convenience.
"""
from __future__ import annotations

import ctypes
import weakref
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgj.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gj.h")

GJ_OK, GJ_ERR_INVALID, GJ_ERR_NOT_ACYCLIC, GJ_ERR_OOM, GJ_ERR_OVERFLOW, GJ_ERR_CUDA, \
    GJ_ERR_TIMEOUT, GJ_ERR_STATE, GJ_ERR_CAPACITY = range(9)
GJ_REL_BORROW, GJ_REL_COPY, GJ_REL_HOST = 0, 1, 2
GJ_OPT_EMIT_ROWS_PER_THREAD = 1
GJ_OPT_TRIANGLE_INTERSECT = 2   # 0 chooses, 1 sorted lists, 2 bitmaps
GJ_OPT_DOWN_COMBINE = 6         # downward pass: 0 combine where links are out of key order, 1 never, 2 always
GJ_OPT_SLOT_ARENA = 7           # bytes of each server slot's bump arena (0: none)
GJ_OPT_SPIN_LIMIT = 3           # failure injection: polls of the group scan's bounded wait
GJ_OPT_TEST_STALL = 4           # failure injection: that wait runs out
GJ_OPT_FAIL_ALLOC_AT = 5        # failure injection: the N-th device allocation fails
SAT = (1 << 64) - 1


class GJError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {_lib.gj_status_str(status).decode()} (status {status})"
        if status in (GJ_ERR_CUDA, GJ_ERR_INVALID):
            last = _lib.gj_last_error().decode()
            if last:
                msg += f" [{last}]"
        super().__init__(msg)


class RelationDesc(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_keys", ctypes.c_int32),
                ("key_attr", ctypes.POINTER(ctypes.c_int32)),
                ("key_cols", ctypes.POINTER(ctypes.c_void_p)),
                ("n_payloads", ctypes.c_int32),
                ("payload_width", ctypes.POINTER(ctypes.c_int32)),
                ("payload_cols", ctypes.POINTER(ctypes.c_void_p)),
                ("flags", ctypes.c_uint32)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("emit_launches", ctypes.c_uint64),
                ("emit_ms", ctypes.c_double), ("emit_rows", ctypes.c_uint64),
                ("emit_bytes", ctypes.c_uint64), ("expand_ms", ctypes.c_double)]


class RequestResult(ctypes.Structure):
    _fields_ = [("total", ctypes.c_uint64), ("status", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("rows", ctypes.c_uint64), ("hash", ctypes.c_uint64),
                ("est_bytes", ctypes.c_uint64), ("t_arrival", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_summary", ctypes.c_double),
                ("t_chunk", ctypes.c_double), ("t_last", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("peak_in_flight", ctypes.c_int32), ("peak_admitted_bytes", ctypes.c_uint64),
                ("wall_s", ctypes.c_double)]


class QuerySizes(ctypes.Structure):
    _fields_ = [("n_rel", ctypes.c_int32), ("n_vars", ctypes.c_int32),
                ("var_attr", ctypes.c_int32 * 64), ("n_cols", ctypes.c_int32),
                ("col_width", ctypes.c_int32 * 64), ("parent", ctypes.c_int32 * 16),
                ("n_groups", ctypes.c_int64 * 16)]


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Loads libgj.so (building it first if the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgj.so not built at {LIB_PATH}")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "gj_status_str": (ctypes.c_char_p, [ctypes.c_int]),
        "gj_version": (ctypes.c_int32, []),
        "gj_last_error": (ctypes.c_char_p, []),
        "gj_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, _P]),
        "gj_destroy": (None, [_P]),
        "gj_set_stream": (ctypes.c_int, [_P, _P]),
        "gj_set_option": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64]),
        "gj_pool_usage": (ctypes.c_int, [_P, _P, _P]),
        "gj_shard_domain": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
        "gj_shard_up": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int64]),
        "gj_shard_down": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int64, _P, _P, _P,
                                         _P, _P]),
        "gj_profile": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Profile)]),
        "gj_load_relation": (ctypes.c_int, [_P, ctypes.POINTER(RelationDesc),
                                            ctypes.POINTER(ctypes.c_int32)]),
        "gj_release_relation": (ctypes.c_int, [_P, ctypes.c_int32]),
        "gj_build_factors": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
        "gj_factor_export": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int64), _P, _P, _P]),
        "gj_query_create": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                           ctypes.POINTER(_P)]),
        "gj_query_create_projected": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                     ctypes.POINTER(_P)]),
        "gj_query_destroy": (None, [_P]),
        "gj_query_sizes": (ctypes.c_int, [_P, ctypes.POINTER(QuerySizes)]),
        "gj_query_set_stream": (ctypes.c_int, [_P, _P]),
        "gj_summarize": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
        "gj_summary_groups": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P]),
        "gj_level": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64,
                                    _P, _P, _P, ctypes.c_uint64,
                                    ctypes.POINTER(ctypes.c_uint64)]),
        "gj_factor_build_noalloc": (ctypes.c_int, [ctypes.c_int32, _P, ctypes.c_int64,
                                                   ctypes.c_int32, ctypes.POINTER(_P),
                                                   ctypes.POINTER(ctypes.c_int32), _P, _P, _P,
                                                   ctypes.POINTER(ctypes.c_int64)]),
        "gj_batch_create": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                           ctypes.POINTER(_P)]),
        "gj_batch_set": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64]),
        "gj_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32)]),
        "gj_batch_run": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
        "gj_batch_destroy": (None, [_P]),
        "gj_server_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.POINTER(_P)]),
        "gj_server_run": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(RequestResult),
                                         ctypes.POINTER(ServerStats)]),
        "gj_server_destroy": (None, [_P]),
        "gj_summary_save": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint64)]),
        "gj_summary_load": (ctypes.c_int, [_P, ctypes.c_char_p, ctypes.POINTER(_P)]),
        "gj_desummarize": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.POINTER(_P), ctypes.POINTER(_P),
                                          ctypes.POINTER(ctypes.c_uint64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_functions() -> list:
    """Names of the functions include/gj.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gj_[a-z_0-9]+)\s*\(", text)))


def _check(st: int, what: str):
    if st != GJ_OK:
        raise GJError(st, what)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _i32(xs):
    arr = (ctypes.c_int32 * max(len(xs), 1))(*xs)
    return arr


class Context:
    """A library context on one device, enqueueing on a torch stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        L = lib()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = _P()
        _check(L.gj_create(ctypes.byref(h), device, _P(stream.cuda_stream)), "gj_create")
        self.h = h
        self._keep = {}
        self._owned = weakref.WeakSet()   # queries, batches, servers on this context

    def _own(self, obj):
        self._owned.add(obj)

    def close(self):
        """Destroys the context; queries, batches and servers still open on
        it are closed first (their handles point into it)."""
        if self.h:
            for obj in list(self._owned):
                obj.close()
            lib().gj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option: int, value: int):
        _check(lib().gj_set_option(self.h, option, value), "gj_set_option")

    def pool_usage(self):
        """(bytes the context's pool has handed out, device allocations made
        since GJ_OPT_FAIL_ALLOC_AT was last set)."""
        used = ctypes.c_uint64()
        n = ctypes.c_int64()
        _check(lib().gj_pool_usage(self.h, ctypes.byref(used), ctypes.byref(n)), "gj_pool_usage")
        return int(used.value), int(n.value)

    def profile(self, enable: bool = True) -> dict:
        """Counters since the last call (synchronises), then profiling on/off."""
        p = Profile()
        _check(lib().gj_profile(self.h, int(enable), ctypes.byref(p)), "gj_profile")
        return {f: getattr(p, f) for f, _ in Profile._fields_}

    def load_relation(self, keys, attrs, payloads=(), flags: int = GJ_REL_BORROW,
                      n_rows: int | None = None) -> int:
        """keys: int32 tensors (device, or host with GJ_REL_HOST); payloads:
        int32 or int64 tensors.  Borrowed tensors are kept alive here."""
        torch = self.torch
        n = int(keys[0].shape[0]) if n_rows is None else n_rows
        kp = (_P * max(len(keys), 1))(*[_ptr(k) for k in keys])
        pp = (_P * max(len(payloads), 1))(*[_ptr(p) for p in payloads])
        widths = [p.element_size() for p in payloads]
        for k in keys:
            assert k.dtype == torch.int32 and k.is_contiguous() and int(k.shape[0]) == n
        for p in payloads:
            assert p.dtype in (torch.int32, torch.int64) and p.is_contiguous()
        aa, ww = _i32(list(attrs)), _i32(widths)
        d = RelationDesc(n, len(keys), ctypes.cast(aa, ctypes.POINTER(ctypes.c_int32)),
                         ctypes.cast(kp, ctypes.POINTER(ctypes.c_void_p)), len(payloads),
                         ctypes.cast(ww, ctypes.POINTER(ctypes.c_int32)),
                         ctypes.cast(pp, ctypes.POINTER(ctypes.c_void_p)), flags)
        rid = ctypes.c_int32()
        _check(lib().gj_load_relation(self.h, ctypes.byref(d), ctypes.byref(rid)),
               "gj_load_relation")
        if flags == GJ_REL_BORROW:
            self._keep[rid.value] = (list(keys), list(payloads))
        return rid.value

    def release_relation(self, rid: int):
        _check(lib().gj_release_relation(self.h, rid), "gj_release_relation")
        self._keep.pop(rid, None)

    def build_factors(self, rid: int, col_order=None):
        co = None if col_order is None else _i32(list(col_order))
        _check(lib().gj_build_factors(self.h, rid, co), "gj_build_factors")

    def factor_export(self, rid: int, n_rows: int, n_keys: int, col_order=None):
        torch = self.torch
        co = None if col_order is None else _i32(list(col_order))
        G = ctypes.c_int64()
        _check(lib().gj_factor_export(self.h, rid, co, ctypes.byref(G), None, None, None),
               "gj_factor_export")
        dev = torch.device("cuda", self.device)
        perm = torch.empty(max(n_rows, 1), dtype=torch.int32, device=dev)
        gstart = torch.empty(G.value + 1, dtype=torch.int32, device=dev)
        gkey = torch.empty(max(n_keys * G.value, 1), dtype=torch.int32, device=dev)
        _check(lib().gj_factor_export(self.h, rid, co, ctypes.byref(G), _P(_ptr(perm)),
                                      _P(_ptr(gstart)), _P(_ptr(gkey))), "gj_factor_export")
        return perm[:n_rows], gstart, gkey[:n_keys * G.value].view(n_keys, G.value)

    def query(self, rel_ids, drop_attrs=()) -> "Query":
        """A query over the loaded relations rel_ids (root first); attributes
        in drop_attrs are projected away early (gj_query_create_projected)."""
        return Query(self, rel_ids, drop_attrs=drop_attrs)


class Query:
    def __init__(self, ctx: Context, rel_ids=None, handle=None, drop_attrs=()):
        self.ctx = ctx
        if handle is not None:
            h = handle
        elif drop_attrs:
            ids = _i32(list(rel_ids))
            drop = _i32(list(drop_attrs))
            h = _P()
            _check(lib().gj_query_create_projected(ctx.h, ids, len(rel_ids), drop, len(drop_attrs),
                                                   ctypes.byref(h)), "gj_query_create_projected")
        else:
            ids = _i32(list(rel_ids))
            h = _P()
            _check(lib().gj_query_create(ctx.h, ids, len(rel_ids), ctypes.byref(h)),
                   "gj_query_create")
        self.h = h
        ctx._own(self)
        s = QuerySizes()
        _check(lib().gj_query_sizes(self.h, ctypes.byref(s)), "gj_query_sizes")
        self.n_rel = s.n_rel
        self.var_attr = list(s.var_attr[:s.n_vars])
        self.col_width = list(s.col_width[:s.n_cols])
        self.parent = list(s.parent[:s.n_rel])
        self.n_groups = list(s.n_groups[:s.n_rel])
        self.total = None
        self.status = None

    def close(self):
        if self.h:
            lib().gj_query_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, path: str) -> int:
        """Stores the summary (gj_summary_save); returns the file size."""
        n = ctypes.c_uint64()
        _check(lib().gj_summary_save(self.h, path.encode(), ctypes.byref(n)), "gj_summary_save")
        return int(n.value)

    @staticmethod
    def load(ctx: "Context", path: str) -> "Query":
        """A query from a stored summary (gj_summary_load)."""
        h = _P()
        _check(lib().gj_summary_load(ctx.h, path.encode(), ctypes.byref(h)), "gj_summary_load")
        q = Query(ctx, handle=h)
        t = ctypes.c_uint64()
        st = lib().gj_summarize(h, ctypes.byref(t))
        q.total = int(t.value)
        q.status = st
        return q

    def set_stream(self, stream):
        """Run this query's later work on its own torch stream."""
        _check(lib().gj_query_set_stream(self.h, _P(stream.cuda_stream)), "gj_query_set_stream")
        self.stream = stream

    def summarize(self) -> int:
        """|Q|; raises GJError on overflow or failure."""
        t = ctypes.c_uint64()
        st = lib().gj_summarize(self.h, ctypes.byref(t))
        self.status = st
        self.total = int(t.value)
        _check(st, "gj_summarize")
        return self.total

    # ---- one rank's part of a row-sharded counting pass (gj_shard_*)
    def children(self, rel: int):
        """rel's children in the join tree, in position order."""
        return [j for j, p in enumerate(self.parent) if p == rel]

    def shard_domain(self, rel: int):
        """(lo, hi) of rel's separator attribute over this rank's rows."""
        lo, hi = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().gj_shard_domain(self.h, rel, ctypes.byref(lo), ctypes.byref(hi)), "gj_shard_domain")
        return int(lo.value), int(hi.value)

    def _children_args(self, rel, msgs):
        ch = self.children(rel)
        ptrs = (_P * max(len(ch), 1))(*[_ptr(msgs[c][0]) for c in ch])
        los = _i32([msgs[c][1] for c in ch] or [0])
        lens = (ctypes.c_int64 * max(len(ch), 1))(*[int(msgs[c][0].numel()) for c in ch])
        return ch, ptrs, los, lens

    def shard_up(self, rel: int, msgs, lo: int = 0, length: int = 1):
        """rel's partial message on this rank (int64 tensor holding uint64
        bits; one entry, the partial join size, for the root).  msgs[c] =
        (global message tensor, lo) of each child c."""
        torch = self.ctx.torch
        dev = torch.device("cuda", self.ctx.device)
        n = 1 if self.parent[rel] < 0 else length
        out = torch.empty(n, dtype=torch.int64, device=dev)
        _, ptrs, los, lens = self._children_args(rel, msgs)
        _check(lib().gj_shard_up(self.h, rel, ptrs, los, lens, _P(_ptr(out)), lo, n), "gj_shard_up")
        return out

    def shard_down(self, rel: int, down, msgs):
        """Partial down messages to rel's children and rel's local partial
        multiplicities, given rel's global down message (tensor, lo) (None
        for the root) and the children's global messages."""
        torch = self.ctx.torch
        dev = torch.device("cuda", self.ctx.device)
        ch, ptrs, los, lens = self._children_args(rel, msgs)
        outs = [torch.empty(int(msgs[c][0].numel()), dtype=torch.int64, device=dev) for c in ch]
        optrs = (_P * max(len(ch), 1))(*[_ptr(o) for o in outs])
        mult = torch.empty(max(self.n_groups[rel], 1), dtype=torch.int64, device=dev)
        dptr, dlo, dlen = (_P(_ptr(down[0])), down[1], int(down[0].numel())) if down is not None else (None, 0, 0)
        _check(lib().gj_shard_down(self.h, rel, dptr, dlo, dlen, ptrs, los, lens, optrs, _P(_ptr(mult))),
               "gj_shard_down")
        return dict(zip(ch, outs)), mult[:self.n_groups[rel]]

    def summary_groups(self, rel: int):
        torch = self.ctx.torch
        G = self.n_groups[rel]
        dev = torch.device("cuda", self.ctx.device)
        w, m, o = (torch.empty(max(G, 1), dtype=torch.int64, device=dev) for _ in range(3))
        _check(lib().gj_summary_groups(self.h, rel, _P(_ptr(w)), _P(_ptr(m)), _P(_ptr(o))),
               "gj_summary_groups")
        self.ctx.stream.synchronize()
        return w[:G], m[:G], o[:G]

    def level(self, level: int, row0: int, n_rows: int, cap: int | None = None):
        torch = self.ctx.torch
        dev = torch.device("cuda", self.ctx.device)
        if cap is None:
            cap = max(1, min(n_rows, (self.total or 0) - row0 if self.total else n_rows))
        val = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        freq = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        off = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        n = ctypes.c_uint64()
        _check(lib().gj_level(self.h, level, row0, n_rows, _P(_ptr(val)), _P(_ptr(freq)),
                              _P(_ptr(off)), cap, ctypes.byref(n)), "gj_level")
        k = int(n.value)
        return val[:k], freq[:k], off[:k]

    def alloc_columns(self, n_rows: int):
        torch = self.ctx.torch
        dev = torch.device("cuda", self.ctx.device)
        return [torch.empty(max(n_rows, 1), dtype=torch.int32 if w == 4 else torch.int64,
                            device=dev) for w in self.col_width]

    def desummarize(self, row0: int, n_rows: int, out=None, rowids: bool = False):
        """Result rows [row0, row0+n_rows) as columns (V keys, then payloads);
        with rowids=True also the row id of every relation.  `out` may be
        device tensors or pinned host tensors (pin_memory): the kernel then
        writes the rows straight into host memory."""
        torch = self.ctx.torch
        if out is None:
            out = self.alloc_columns(n_rows)
        cols = (_P * len(out))(*[_ptr(t) for t in out])
        rid_t = None
        rid = None
        if rowids:
            dev = torch.device("cuda", self.ctx.device)
            rid_t = [torch.empty(max(n_rows, 1), dtype=torch.int32, device=dev)
                     for _ in range(self.n_rel)]
            rid = (_P * self.n_rel)(*[_ptr(t) for t in rid_t])
        n = ctypes.c_uint64()
        _check(lib().gj_desummarize(self.h, row0, n_rows, cols, rid, ctypes.byref(n)),
               "gj_desummarize")
        k = int(n.value)
        res = [t[:k] for t in out]
        if rowids:
            return res, [t[:k] for t in rid_t]
        return res


GJ_BATCH_GRID_MULT = 1


class Batch:
    """Many queries summarised together (gj_batch_*)."""

    def __init__(self, ctx: Context, queries_rel_ids):
        self.ctx = ctx
        flat = [r for q in queries_rel_ids for r in q]
        off = [0]
        for q in queries_rel_ids:
            off.append(off[-1] + len(q))
        h = _P()
        _check(lib().gj_batch_create(ctx.h, _i32(flat), _i32(off), len(queries_rel_ids),
                                     ctypes.byref(h)), "gj_batch_create")
        self.h = h
        ctx._own(self)
        self.n_queries = len(queries_rel_ids)
        n = ctypes.c_int64()
        r, l, kb = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().gj_batch_info(h, ctypes.byref(n), ctypes.byref(r), ctypes.byref(l),
                                   ctypes.byref(kb)), "gj_batch_info")
        self.n_rows, self.n_relations, self.levels, self.key_bits = n.value, r.value, l.value, kb.value
        torch = ctx.torch
        dev = torch.device("cuda", ctx.device)
        self.totals = torch.zeros(self.n_queries, dtype=torch.int64, device=dev)
        self.status = torch.zeros(self.n_queries, dtype=torch.int32, device=dev)

    def set_grid_mult(self, m: int):
        _check(lib().gj_batch_set(self.h, GJ_BATCH_GRID_MULT, m), "gj_batch_set")

    def run(self, use_graph: bool = True):
        """Enqueue the batch (no synchronisation); results in .totals/.status."""
        _check(lib().gj_batch_run(self.h, int(use_graph), _P(_ptr(self.totals)),
                                  _P(_ptr(self.status))), "gj_batch_run")

    def close(self):
        if self.h:
            lib().gj_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NativeServer:
    """The native serving runtime (gj_server_*): replays arrival traces."""

    def __init__(self, ctx: Context, n_slots: int = 16, hbm_budget: int = 150 * 10**9,
                 chunk_rows: int = 1 << 20, max_rows: int = 0):
        """max_rows: result rows streamed per request (0: the whole result),
        in chunks of chunk_rows."""
        self.ctx = ctx
        h = _P()
        _check(lib().gj_server_create(ctx.h, n_slots, hbm_budget, chunk_rows, max_rows, ctypes.byref(h)),
               "gj_server_create")
        self.h = h
        ctx._own(self)

    def run(self, queries_rel_ids, arrival_offsets):
        """queries_rel_ids[i] arrives arrival_offsets[i] s after the start.
        Returns (list of result dicts, stats dict)."""
        n = len(queries_rel_ids)
        flat = [r for q in queries_rel_ids for r in q]
        off = [0]
        for q in queries_rel_ids:
            off.append(off[-1] + len(q))
        arr = (ctypes.c_double * max(n, 1))(*[float(x) for x in arrival_offsets])
        res = (RequestResult * max(n, 1))()
        st = ServerStats()
        _check(lib().gj_server_run(self.h, n, _i32(flat), _i32(off), arr, res, ctypes.byref(st)),
               "gj_server_run")
        out = [{f: getattr(res[i], f) for f, _ in RequestResult._fields_} for i in range(n)]
        return out, {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            lib().gj_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_query(ctx: Context, query, flags: int = GJ_REL_BORROW) -> list:
    """Registers every relation of a datagen.Query (numpy columns) and returns
    their ids, root first.  Columns are copied to the context's device."""
    torch = ctx.torch
    dev = torch.device("cuda", ctx.device)
    ids = []
    for R in query.relations:
        keys = [torch.from_numpy(k).to(dev) for k in R.keys]
        pays = [torch.from_numpy(p).to(dev) for p in R.payloads]
        ids.append(ctx.load_relation(keys, R.attrs, pays, flags=flags, n_rows=R.n_rows))
    return ids
