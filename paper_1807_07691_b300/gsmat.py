"""ctypes binding of libgsmat (include/gsmat.h): argument marshalling only.

Every step of loading and querying runs in the library's CUDA kernels; this
module converts Python/numpy/torch arguments to the C ABI and back.  If the
shared library is missing the import fails loudly -- there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsmat.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "gsmat.h")

OK = 0
ERR_INVALID_ARG = 1
ERR_UNSUPPORTED = 2
ERR_OOM = 3
ERR_CAPACITY = 4
ERR_CUDA = 5
ERR_DEVICE_CHECK = 6

SORTED = 0
PLAN_ORDER = 1
COUNT_ONLY = 2
NO_INTERSECT = 4
PLAN_COST = 8
PLAN_COST_MAX = 8

STEP_CROSS, STEP_EXPAND_S, STEP_EXPAND_O, STEP_FILTER = 0, 1, 2, 3
MAX_PATTERNS = 64


class GsmatError(RuntimeError):
    def __init__(self, code: int, detail: str = ""):
        self.code = code
        self.detail = detail
        super().__init__(f"gsmat error {code} ({_strerror(code)}): {detail}")


class Pattern(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("p", ctypes.c_int32), ("o", ctypes.c_int32),
                ("s_var", ctypes.c_uint8), ("p_var", ctypes.c_uint8), ("o_var", ctypes.c_uint8),
                ("_pad", ctypes.c_uint8)]


class StoreInfo(ctypes.Structure):
    _fields_ = [("n_input", ctypes.c_int64), ("n_unique", ctypes.c_int64), ("n_predicates", ctypes.c_int32),
                ("max_entity", ctypes.c_int32), ("max_predicate", ctypes.c_int32),
                ("n_dense_rows_s", ctypes.c_int32), ("n_dense_rows_o", ctypes.c_int32),
                ("_reserved", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


class PredStats(ctypes.Structure):
    _fields_ = [("pred_id", ctypes.c_int32), ("nnz", ctypes.c_int32), ("nr_s", ctypes.c_int32),
                ("nr_o", ctypes.c_int32)]


class QueryStats(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("order", ctypes.c_int32 * MAX_PATTERNS),
                ("kind", ctypes.c_int32 * MAX_PATTERNS), ("est_rows", ctypes.c_double * MAX_PATTERNS),
                ("rows", ctypes.c_int64 * MAX_PATTERNS), ("est_cost", ctypes.c_double),
                ("result_rows", ctypes.c_int64)]


class BGPStruct(ctypes.Structure):
    _fields_ = [("pats", ctypes.c_void_p), ("n_pats", ctypes.c_int32), ("n_vars", ctypes.c_int32)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("arena_bytes", ctypes.c_int64),
                ("max_rows", ctypes.c_int64), ("use_graph", ctypes.c_int32), ("compact_results", ctypes.c_int32),
                ("reorder_mode", ctypes.c_int32), ("plan_cost", ctypes.c_int32), ("expand_slots", ctypes.c_int32),
                ("_pad", ctypes.c_int32)]


class BatchStats(ctypes.Structure):
    _fields_ = [("n_queries", ctypes.c_int32), ("n_in_kernel", ctypes.c_int32), ("n_reordered", ctypes.c_int32),
                ("n_fallback", ctypes.c_int32), ("kernel_ms", ctypes.c_double), ("reorder_ms", ctypes.c_double),
                ("arena_used", ctypes.c_int64),
                ("block", ctypes.c_int32), ("grid", ctypes.c_int32), ("n_intersect", ctypes.c_int32),
                ("_pad", ctypes.c_int32)]


class Tiles(ctypes.Structure):
    _fields_ = [("expand_items", ctypes.c_int32), ("short_row", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("slots", ctypes.c_int32), ("budget_bytes", ctypes.c_int64),
                ("batch", BatchConfig), ("batch_lone", ctypes.c_int32), ("lanes", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "batches", "fallbacks", "queued",
                                              "in_flight", "in_flight_bytes", "direct")]


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("algo_bytes", ctypes.c_double), ("items", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgsmat.so is not built ({LIB_PATH}); run python -m paper_1807_07691_b300.build")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    c_int = ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "gsmat_strerror": ([c_int], ctypes.c_char_p),
        "gsmat_last_error": ([], ctypes.c_char_p),
        "gsmat_version": ([], c_int),
        "gsmat_set_allocator": ([vp, vp, vp], c_int),
        "gsmat_load": ([vp, i64, c_int, vp, P(vp)], c_int),
        "gsmat_store_info": ([vp, P(StoreInfo)], c_int),
        "gsmat_store_pred_stats": ([vp, vp, i32, P(i32)], c_int),
        "gsmat_store_export": ([vp, i32, c_int, vp, vp, vp, vp], c_int),
        "gsmat_store_pred_index": ([vp, i32], i32),
        "gsmat_store_free": ([vp], None),
        "gsmat_query": ([vp, vp, c_int, c_int, u32, vp, P(vp)], c_int),
        "gsmat_table_info": ([vp, P(i64), P(i32), vp], c_int),
        "gsmat_table_column": ([vp, i32, P(vp)], c_int),
        "gsmat_table_copy": ([vp, vp, c_int, vp], c_int),
        "gsmat_table_copy_async": ([vp, vp, c_int, vp], c_int),
        "gsmat_table_stats": ([vp, P(QueryStats)], c_int),
        "gsmat_table_free": ([vp], None),
        "gsmat_plan": ([vp, c_int, c_int, vp, vp, vp, vp, vp], c_int),
        "gsmat_plan_cost": ([vp, c_int, c_int, vp, vp, vp, vp, vp], c_int),
        "gsmat_table_project": ([vp, vp, i32, c_int, vp, P(vp)], c_int),
        "gsmat_query_shard": ([vp, vp, c_int, c_int, u32, i32, i32, vp, P(vp)], c_int),
        "gsmat_table_merge": ([vp, i32, vp, P(vp)], c_int),
        "gsmat_dict_create": ([P(vp)], c_int),
        "gsmat_dict_free": ([vp], None),
        "gsmat_dict_add_text": ([vp, ctypes.c_char_p, i64, P(i64)], c_int),
        "gsmat_dict_set_threads": ([vp, i32], c_int),
        "gsmat_dict_triples": ([vp, P(vp), P(i64)], c_int),
        "gsmat_dict_size": ([vp, P(i32), P(i32)], c_int),
        "gsmat_dict_lookup": ([vp, c_int, ctypes.c_char_p, i64, P(i32)], c_int),
        "gsmat_dict_decode": ([vp, c_int, vp, i64, vp, vp], c_int),
        "gsmat_sparql_parse": ([vp, ctypes.c_char_p, i64, P(vp)], c_int),
        "gsmat_sparql_info": ([vp, P(vp), P(i32), P(i32), P(vp), P(i32), P(i32)], c_int),
        "gsmat_sparql_var_name": ([vp, i32], ctypes.c_char_p),
        "gsmat_sparql_free": ([vp], None),
        "gsmat_batch_prepare": ([vp, vp, i32, vp, vp, P(vp)], c_int),
        "gsmat_batch_execute": ([vp, vp], c_int),
        "gsmat_batch_result": ([vp, i32, P(i64), P(i32), P(i32)], c_int),
        "gsmat_batch_column": ([vp, i32, i32, P(vp)], c_int),
        "gsmat_batch_copy": ([vp, i32, vp, c_int, vp], c_int),
        "gsmat_batch_stats": ([vp, vp], c_int),
        "gsmat_batch_free": ([vp], None),
        "gsmat_batch_autotune": ([vp, vp, i32, vp, vp, vp], c_int),
        "gsmat_server_create": ([vp, vp, P(vp)], c_int),
        "gsmat_server_submit": ([vp, vp, c_int, c_int, P(i64)], c_int),
        "gsmat_server_wait": ([vp, i64, i64, P(i32)], c_int),
        "gsmat_server_result": ([vp, i64, P(i64), P(i32), P(ctypes.c_double)], c_int),
        "gsmat_server_copy": ([vp, i64, vp, c_int, vp], c_int),
        "gsmat_server_release": ([vp, i64], c_int),
        "gsmat_server_stats": ([vp, vp], c_int),
        "gsmat_server_destroy": ([vp], None),
        "gsmat_radix_sort_u64": ([vp, vp, i64, c_int, c_int, vp], c_int),
        "gsmat_sort_rows": ([vp, c_int, c_int, c_int, i64, vp, u32, vp], c_int),
        "gsmat_exclusive_scan_i32": ([vp, vp, i64, vp], c_int),
        "gsmat_exclusive_scan_i32_noalloc": ([vp, vp, i64, vp], c_int),
        "gsmat_exclusive_scan_i32_noalloc_max": ([], i64),
        "gsmat_selftest_wait_expiry": ([i32, vp], c_int),
        "gsmat_store_set_tiles": ([vp, vp], c_int),
        "gsmat_store_get_tiles": ([vp, vp], c_int),
        "gsmat_store_tune": ([vp, vp, i32, vp, vp], c_int),
        "gsmat_profile_enable": ([c_int], c_int),
        "gsmat_profile_read": ([vp, i32, P(i32), c_int], c_int),
        "gsmat_launch_count": ([], i64),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


_lib = _load()


def lib():
    return _lib


def header_functions() -> list:
    """Names of the functions declared in include/gsmat.h."""
    with open(HEADER_PATH) as f:
        text = f.read()
    return sorted(set(re.findall(r"GSMAT_API\s+[\w\s\*]+?\b(gsmat_\w+)\s*\(", text)))


def _strerror(code: int) -> str:
    return _lib.gsmat_strerror(code).decode()


def _check(rc: int):
    if rc != OK:
        raise GsmatError(rc, _lib.gsmat_last_error().decode())


def _stream_ptr(stream):
    """A cudaStream_t from None (torch's current stream if CUDA is up, else
    the legacy default stream), an int, or a torch.cuda.Stream."""
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _patterns(bgp):
    """(ctypes array of Pattern, n, n_vars) from a BGP-like object, an (n, 6)
    array (s, p, o, s_var, p_var, o_var) or a list of (s, p, o, s_var,
    o_var) tuples."""
    n_vars = getattr(bgp, "n_vars", None)
    if hasattr(bgp, "as_array"):
        arr = bgp.as_array()
    else:
        arr = np.asarray(bgp, dtype=np.int64)
        if arr.ndim == 2 and arr.shape[1] == 5:
            arr = np.stack([arr[:, 0], arr[:, 1], arr[:, 2], arr[:, 3], np.zeros(len(arr), np.int64), arr[:, 4]], 1)
    arr = arr.reshape(-1, 6)
    pats = (Pattern * max(1, arr.shape[0]))()
    for i, (s, p, o, sv, pv, ov) in enumerate(arr.tolist()):
        pats[i] = Pattern(int(s), int(p), int(o), int(sv), int(pv), int(ov), 0)
    return pats, arr.shape[0], n_vars


# ----------------------------------------------------------------------------


class Table:
    """A device-resident binding table (columns are int32 device arrays)."""

    def __init__(self, handle):
        self._h = handle

    def __del__(self):
        self.free()

    def free(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.gsmat_table_free(h)
        self._h = None

    @property
    def shape(self):
        rows, cols = ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.gsmat_table_info(self._h, ctypes.byref(rows), ctypes.byref(cols), None))
        return int(rows.value), int(cols.value)

    @property
    def rows(self) -> int:
        return self.shape[0]

    @property
    def col_vars(self) -> list:
        rows, cols = self.shape
        buf = (ctypes.c_int32 * max(1, cols))()
        _check(_lib.gsmat_table_info(self._h, None, None, buf))
        return [int(buf[i]) for i in range(cols)]

    def column_ptr(self, c: int) -> int:
        p = ctypes.c_void_p()
        _check(_lib.gsmat_table_column(self._h, c, ctypes.byref(p)))
        return p.value or 0

    def to_numpy(self, stream=None) -> np.ndarray:
        rows, cols = self.shape
        out = np.empty((rows, cols), dtype=np.int32)
        if rows and cols:
            _check(_lib.gsmat_table_copy(self._h, out.ctypes.data, 0, _stream_ptr(stream)))
        return out

    def copy_to(self, dst, stream=None, sync: bool = True):
        """Copy the table row-major into dst: a host numpy array or a host
        (ideally pinned) / CUDA torch tensor of int32 with rows*cols
        elements.  sync=False only enqueues the copy on `stream`
        (gsmat_table_copy_async): keep the table and dst alive until the
        stream has passed it."""
        rows, cols = self.shape
        if rows == 0 or cols == 0:
            return dst
        fn = _lib.gsmat_table_copy if sync else _lib.gsmat_table_copy_async
        if hasattr(dst, "data_ptr"):
            import torch

            if dst.dtype != torch.int32 or not dst.is_contiguous() or dst.numel() < rows * cols:
                raise ValueError("destination must be a contiguous int32 tensor of rows*cols elements")
            _check(fn(self._h, ctypes.c_void_p(dst.data_ptr()), 1 if dst.is_cuda else 0, _stream_ptr(stream)))
        else:
            if dst.size < rows * cols or dst.dtype != np.int32 or not dst.flags.c_contiguous:
                raise ValueError("destination must be a contiguous int32 array of rows*cols elements")
            _check(fn(self._h, dst.ctypes.data, 0, _stream_ptr(stream)))
        return dst

    def to_torch(self, stream=None):
        """Row-major (rows, cols) int32 CUDA tensor (a copy)."""
        import torch

        rows, cols = self.shape
        out = torch.empty((rows, cols), dtype=torch.int32, device="cuda")
        if rows and cols:
            _check(_lib.gsmat_table_copy(self._h, ctypes.c_void_p(out.data_ptr()), 1, _stream_ptr(stream)))
        return out

    def project(self, variables, distinct: bool = False, stream=None) -> "Table":
        """gsmat_table_project: the given variables' columns, rows ascending
        (each once with ``distinct``), as a new device table."""
        v = np.ascontiguousarray(np.asarray(list(variables), dtype=np.int32))
        h = ctypes.c_void_p()
        _check(_lib.gsmat_table_project(self._h, v.ctypes.data, int(v.size), 1 if distinct else 0,
                                        _stream_ptr(stream), ctypes.byref(h)))
        return Table(h)

    def stats(self) -> dict:
        s = QueryStats()
        _check(_lib.gsmat_table_stats(self._h, ctypes.byref(s)))
        n = s.n_steps
        return {
            "order": [s.order[i] for i in range(n)],
            "kind": [s.kind[i] for i in range(n)],
            "est_rows": [s.est_rows[i] for i in range(n)],
            "rows": [int(s.rows[i]) for i in range(n)],
            "est_cost": s.est_cost,
            "result_rows": int(s.result_rows),
        }


class Store:
    """The device-resident SM store built by gsmat_load."""

    def __init__(self, triples, stream=None):
        h = ctypes.c_void_p()
        on_device = 0
        keep = None
        if hasattr(triples, "data_ptr"):  # torch tensor
            import torch

            t = triples
            if t.dtype != torch.int32 or t.dim() != 2 or t.shape[1] != 3 or not t.is_contiguous():
                raise ValueError("triples must be a contiguous (n, 3) int32 tensor")
            ptr, n = t.data_ptr(), t.shape[0]
            on_device = 1 if t.is_cuda else 0
            keep = t
        else:
            arr = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
            ptr, n = arr.ctypes.data, arr.shape[0]
            keep = arr
        _check(_lib.gsmat_load(ctypes.c_void_p(ptr), n, on_device, _stream_ptr(stream), ctypes.byref(h)))
        del keep
        self._h = h

    def __del__(self):
        self.free()

    def free(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.gsmat_store_free(h)
        self._h = None

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = StoreInfo()
        _check(_lib.gsmat_store_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in StoreInfo._fields_ if not f.startswith("_")}

    def pred_stats(self) -> list:
        n = self.info()["n_predicates"]
        buf = (PredStats * max(1, n))()
        got = ctypes.c_int32()
        _check(_lib.gsmat_store_pred_stats(self._h, buf, n, ctypes.byref(got)))
        return [{"pred_id": b.pred_id, "nnz": b.nnz, "nr_s": b.nr_s, "nr_o": b.nr_o} for b in buf[: got.value]]

    def pred_index(self, pred_id: int) -> int:
        return int(_lib.gsmat_store_pred_index(self._h, int(pred_id)))

    def export(self, pred_id: int, side: int, stream=None):
        """(row_ids, row_ptr, entries) of one predicate on one side (host)."""
        st = {s["pred_id"]: s for s in self.pred_stats()}[int(pred_id)]
        nr = st["nr_s"] if side == 0 else st["nr_o"]
        rid = np.empty(max(1, nr), np.int32)
        ptr = np.empty(nr + 1, np.int64)
        ent = np.empty(max(1, st["nnz"]), np.int32)
        _check(_lib.gsmat_store_export(self._h, int(pred_id), int(side), rid.ctypes.data, ptr.ctypes.data,
                                       ent.ctypes.data, _stream_ptr(stream)))
        return rid[:nr], ptr, ent[: st["nnz"]]

    def tiles(self) -> dict:
        """The store's tile shapes (gsmat_store_get_tiles)."""
        t = Tiles()
        _check(_lib.gsmat_store_get_tiles(self._h, ctypes.byref(t)))
        return {"expand_items": t.expand_items, "short_row": t.short_row}

    def set_tiles(self, expand_items: int = 2048, short_row: int = 64):
        t = Tiles(int(expand_items), int(short_row))
        _check(_lib.gsmat_store_set_tiles(self._h, ctypes.byref(t)))

    def tune(self, bgps, stream=None) -> dict:
        """Autotune the tile shapes on a sample of BGPs (gsmat_store_tune);
        the fastest is kept on the store and returned."""
        arr, keep = _bgp_array(bgps)
        t = Tiles()
        _check(_lib.gsmat_store_tune(self._h, arr, len(bgps), _stream_ptr(stream), ctypes.byref(t)))
        return {"expand_items": t.expand_items, "short_row": t.short_row}

    @staticmethod
    def marshal(bgp, n_vars=None):
        """Pre-converted arguments for query_raw: (patterns, n, n_vars)."""
        pats, n, nv = _patterns(bgp)
        if n_vars is None:
            n_vars = nv
        if n_vars is None:
            raise ValueError("n_vars is required")
        return pats, n, int(n_vars)

    def query_raw(self, marshalled, flags: int = SORTED, stream=None) -> Table:
        pats, n, nv = marshalled
        h = ctypes.c_void_p()
        _check(_lib.gsmat_query(self._h, pats, n, nv, flags, _stream_ptr(stream), ctypes.byref(h)))
        return Table(h)

    def query(self, bgp, n_vars=None, flags: int = SORTED, stream=None) -> Table:
        return self.query_raw(self.marshal(bgp, n_vars), flags, stream)

    def query_shard(self, bgp, shard: int, n_shards: int, n_vars=None, flags: int = SORTED, stream=None) -> Table:
        """gsmat_query_shard: the part of the result that derives from the
        shard-th of n_shards contiguous parts of the first plan step."""
        pats, n, nv = self.marshal(bgp, n_vars)
        h = ctypes.c_void_p()
        _check(_lib.gsmat_query_shard(self._h, pats, n, nv, flags, int(shard), int(n_shards), _stream_ptr(stream),
                                      ctypes.byref(h)))
        return Table(h)

    def sparql(self, query, dictionary: "Dictionary | None" = None, flags: int = SORTED, stream=None) -> Table:
        """Evaluate SPARQL text (or a parsed Sparql): the BGP by gsmat_query,
        then the projection / DISTINCT by gsmat_table_project when the
        query asks for anything but all variables in order."""
        q = query if isinstance(query, Sparql) else Sparql(query, dictionary)
        T = self.query(q, flags=flags & ~PLAN_ORDER, stream=stream)
        if q.projection == list(range(q.n_vars)) and not q.distinct:
            return T
        P = T.project(q.projection, q.distinct, stream=stream)
        T.free()
        return P


def merge_tables(tables, stream=None) -> Table:
    """gsmat_table_merge: the rows of tables with the same columns, together,
    ascending (e.g. the sorted shards of one query)."""
    arr = (ctypes.c_void_p * len(tables))(*[t._h.value for t in tables])
    h = ctypes.c_void_p()
    _check(_lib.gsmat_table_merge(arr, len(tables), _stream_ptr(stream), ctypes.byref(h)))
    return Table(h)


def gather_rows(rows: np.ndarray, dst: int = 0, group=None):
    """Host side of row sharding across ranks: rank r passes the rows of
    shard r (int32, rows x cols, e.g. gsmat_query_shard with
    GSMAT_PLAN_ORDER copied to the host); rank `dst` returns all of them
    back to back in rank order -- for plan-order shards, the full plan-order
    result -- and the other ranks return None.  Uses torch.distributed
    object collectives (any backend)."""
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    parts = [None] * world if rank == dst else None
    dist.gather_object(np.ascontiguousarray(rows, dtype=np.int32), parts, dst=dst, group=group)
    if rank != dst:
        return None
    return np.concatenate([p.reshape(-1, rows.shape[1]) for p in parts], axis=0)


def gather_shards(rows, dst: int = 0, group=None):
    """Row sharding across ranks with tensor collectives: rank r passes the
    rows of shard r as a (rows, cols) int32 tensor (e.g. ``Table.to_torch()``
    of ``query_shard`` in plan order, a device tensor under NCCL, a host one
    under gloo); rank `dst` returns every rank's rows back to back in rank
    order -- for plan-order shards, the full plan-order result -- and the
    other ranks return None.  The shard sizes are exchanged first, then each
    shard, padded to the largest, is all-gathered on the tensors' device:
    the rows never pass through host objects."""
    import torch
    import torch.distributed as dist

    if rows.dim() != 2:
        raise ValueError("gather_shards: rows must be a (rows, cols) tensor")
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    n, c = rows.shape
    shape = torch.tensor([n, c], dtype=torch.int64, device=rows.device)
    shapes = [torch.empty_like(shape) for _ in range(world)]
    dist.all_gather(shapes, shape, group=group)
    ns = [int(x[0]) for x in shapes]
    if len({int(x[1]) for x in shapes}) != 1:
        raise ValueError("gather_shards: the shards have different column counts")
    m = max(ns)
    if m == 0 or c == 0:
        return rows.new_empty((sum(ns), c)) if rank == dst else None
    buf = rows.new_zeros((m, c))
    buf[:n] = rows
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    if rank != dst:
        return None
    return torch.cat([part[:k] for part, k in zip(parts, ns)], dim=0)


# ----------------------------------------------------------------------------


def _text_bytes(text) -> bytes:
    return text.encode("utf-8") if isinstance(text, str) else bytes(text)


class Dictionary:
    """h_p and h_so by first occurrence (gsmat_dict_*; Sec. 5.2)."""

    SO = 0
    P = 1

    def __init__(self, text=None, threads: int = 0):
        h = ctypes.c_void_p()
        _check(_lib.gsmat_dict_create(ctypes.byref(h)))
        self._h = h
        if threads:
            self.set_threads(threads)
        if text is not None:
            self.add_text(text)

    def set_threads(self, n: int):
        """Host threads numbering the terms (0: automatic); codes do not
        depend on it."""
        _check(_lib.gsmat_dict_set_threads(self._h, int(n)))

    def __del__(self):
        self.free()

    def free(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.gsmat_dict_free(h)
        self._h = None

    @property
    def handle(self):
        return self._h

    def add_text(self, text) -> int:
        b = _text_bytes(text)
        n = ctypes.c_int64()
        _check(_lib.gsmat_dict_add_text(self._h, b, len(b), ctypes.byref(n)))
        return int(n.value)

    def triples(self) -> np.ndarray:
        """(n, 3) int32 (s, p, o) codes of everything added (a copy)."""
        p, n = ctypes.c_void_p(), ctypes.c_int64()
        _check(_lib.gsmat_dict_triples(self._h, ctypes.byref(p), ctypes.byref(n)))
        if n.value == 0:
            return np.zeros((0, 3), np.int32)
        arr = (ctypes.c_int32 * (3 * n.value)).from_address(p.value)
        return np.frombuffer(arr, dtype=np.int32).reshape(-1, 3).copy()

    def size(self) -> tuple:
        np_, nt = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.gsmat_dict_size(self._h, ctypes.byref(np_), ctypes.byref(nt)))
        return int(np_.value), int(nt.value)

    def lookup(self, term: str, kind: int = 0) -> int:
        b = _text_bytes(term)
        c = ctypes.c_int32()
        _check(_lib.gsmat_dict_lookup(self._h, kind, b, len(b), ctypes.byref(c)))
        return int(c.value)

    def decode(self, codes, kind: int = 0) -> list:
        c = np.ascontiguousarray(np.asarray(codes, dtype=np.int32).ravel())
        n = int(c.size)
        terms = (ctypes.c_char_p * max(1, n))()
        lens = np.zeros(max(1, n), np.int32)
        _check(_lib.gsmat_dict_decode(self._h, kind, c.ctypes.data, n, ctypes.cast(terms, ctypes.c_void_p),
                                      lens.ctypes.data))
        return [ctypes.string_at(terms[i], int(lens[i])).decode("utf-8") for i in range(n)]

    def decode_rows(self, rows) -> list:
        """Rows of a result (subject/object codes) as tuples of terms."""
        rows = np.asarray(rows, dtype=np.int32)
        if rows.size == 0:
            return [tuple() for _ in range(rows.shape[0])]
        flat = self.decode(rows.ravel(), self.SO)
        k = rows.shape[1]
        return [tuple(flat[i * k:(i + 1) * k]) for i in range(rows.shape[0])]


class Sparql:
    """A parsed SPARQL query (gsmat_sparql_*): usable wherever a BGP is."""

    def __init__(self, text, dictionary: Dictionary | None = None):
        b = _text_bytes(text)
        h = ctypes.c_void_p()
        _check(_lib.gsmat_sparql_parse(dictionary.handle if dictionary is not None else None, b, len(b),
                                       ctypes.byref(h)))
        self._h = h
        pats, n, nv, proj, nproj, dist = (ctypes.c_void_p(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_void_p(),
                                          ctypes.c_int32(), ctypes.c_int32())
        _check(_lib.gsmat_sparql_info(h, ctypes.byref(pats), ctypes.byref(n), ctypes.byref(nv), ctypes.byref(proj),
                                      ctypes.byref(nproj), ctypes.byref(dist)))
        arr = (Pattern * n.value).from_address(pats.value)
        self.patterns = [(p.s, p.p, p.o, p.s_var, p.o_var) for p in arr]
        self.n_vars = int(nv.value)
        pr = (ctypes.c_int32 * max(1, nproj.value)).from_address(proj.value) if nproj.value else []
        self.projection = [int(pr[i]) for i in range(nproj.value)]
        self.distinct = bool(dist.value)
        self.var_names = [_lib.gsmat_sparql_var_name(h, v).decode("utf-8") for v in range(self.n_vars)]
        _lib.gsmat_sparql_free(h)
        self._h = None

    def as_array(self) -> np.ndarray:
        a = np.zeros((len(self.patterns), 6), np.int64)
        for i, (s, p, o, sv, ov) in enumerate(self.patterns):
            a[i] = (s, p, o, sv, 0, ov)
        return a


# ----------------------------------------------------------------------------


def _config(cfg):
    if cfg is None:
        return None
    c = BatchConfig()
    c.block = int(cfg.get("block", 0))
    c.ctas_per_sm = int(cfg.get("ctas_per_sm", 0))
    c.arena_bytes = int(cfg.get("arena_bytes", 0))
    c.max_rows = int(cfg.get("max_rows", 0))
    c.use_graph = int(cfg.get("use_graph", 1))
    c.compact_results = int(cfg.get("compact_results", 0))
    c.reorder_mode = int(cfg.get("reorder_mode", 0))
    c.plan_cost = int(cfg.get("plan_cost", 0))
    c.expand_slots = int(cfg.get("expand_slots", 0))
    return c


def _bgp_array(bgps, n_vars_list=None):
    """(BGPStruct array, keep-alive list) from BGP-like objects."""
    keep = []
    arr = (BGPStruct * len(bgps))()
    for i, q in enumerate(bgps):
        pats, n, nv = _patterns(q)
        if n_vars_list is not None:
            nv = n_vars_list[i]
        if nv is None:
            raise ValueError("n_vars is required")
        keep.append(pats)
        arr[i] = BGPStruct(ctypes.cast(pats, ctypes.c_void_p), n, int(nv))
    return arr, keep


class Batch:
    """A prepared batch of BGPs run by the persistent kernel (gsmat_batch_*)."""

    def __init__(self, store: "Store", bgps, config: dict | None = None, stream=None, n_vars_list=None):
        self._arr, self._keep = _bgp_array(bgps, n_vars_list)
        self.n = len(bgps)
        self._store = store  # the store must outlive the batch
        cfg = _config(config)
        h = ctypes.c_void_p()
        _check(_lib.gsmat_batch_prepare(store.handle, self._arr, self.n, ctypes.byref(cfg) if cfg else None,
                                        _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        self.free()

    def free(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.gsmat_batch_free(h)
        self._h = None

    def execute(self, stream=None):
        _check(_lib.gsmat_batch_execute(self._h, _stream_ptr(stream)))
        return self

    def result(self, i: int):
        rows, cols, path = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.gsmat_batch_result(self._h, i, ctypes.byref(rows), ctypes.byref(cols), ctypes.byref(path)))
        return int(rows.value), int(cols.value), int(path.value)

    def to_numpy(self, i: int, stream=None) -> np.ndarray:
        rows, cols, _ = self.result(i)
        out = np.empty((rows, cols), dtype=np.int32)
        if rows and cols:
            _check(_lib.gsmat_batch_copy(self._h, i, out.ctypes.data, 0, _stream_ptr(stream)))
        return out

    def copy_to(self, i: int, dst, stream=None):
        """Copy result i row-major into dst (a contiguous int32 numpy array
        or torch tensor, host or CUDA, of at least rows*cols elements)."""
        rows, cols, _ = self.result(i)
        if rows and cols:
            if hasattr(dst, "data_ptr"):
                import torch

                if dst.dtype != torch.int32 or not dst.is_contiguous() or dst.numel() < rows * cols:
                    raise ValueError("destination must be a contiguous int32 tensor of rows*cols elements")
                on_dev, ptr = (1 if dst.is_cuda else 0), dst.data_ptr()
            else:
                if dst.dtype != np.int32 or not dst.flags.c_contiguous or dst.size < rows * cols:
                    raise ValueError("destination must be a contiguous int32 array of rows*cols elements")
                on_dev, ptr = 0, dst.ctypes.data
            _check(_lib.gsmat_batch_copy(self._h, i, ctypes.c_void_p(ptr), on_dev, _stream_ptr(stream)))
        return dst

    def stats(self) -> dict:
        s = BatchStats()
        _check(_lib.gsmat_batch_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in BatchStats._fields_}


class Server:
    """Continuous-batching server over a resident store (gsmat_server_*)."""

    def __init__(self, store: "Store", max_batch: int = 0, slots: int = 0, budget_bytes: int = 0,
                 batch: dict | None = None, batch_lone: bool = False, lanes: int = 0):
        c = ServerConfig()
        c.max_batch = max_batch
        c.slots = slots
        c.budget_bytes = budget_bytes
        c.batch_lone = 1 if batch_lone else 0
        c.lanes = lanes
        bc = _config(batch)
        if bc is not None:
            c.batch = bc
        self._store = store  # must outlive the server
        h = ctypes.c_void_p()
        _check(_lib.gsmat_server_create(store.handle, ctypes.byref(c), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.gsmat_server_destroy(h)
        self._h = None

    @staticmethod
    def marshal(bgp, n_vars=None):
        """Pre-converted arguments for submit_raw (saves the conversion on a
        hot submission path)."""
        pats, n, nv = _patterns(bgp)
        return pats, n, int(nv if n_vars is None else n_vars)

    def submit_raw(self, marshalled) -> int:
        pats, n, nv = marshalled
        t = ctypes.c_int64()
        _check(_lib.gsmat_server_submit(self._h, pats, n, nv, ctypes.byref(t)))
        return int(t.value)

    def submit(self, bgp, n_vars=None) -> int:
        return self.submit_raw(self.marshal(bgp, n_vars))

    def wait(self, ticket: int, timeout_us: int = -1) -> bool:
        done = ctypes.c_int32()
        _check(_lib.gsmat_server_wait(self._h, ticket, timeout_us, ctypes.byref(done)))
        return bool(done.value)

    def result(self, ticket: int):
        rows, cols, lat = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
        _check(_lib.gsmat_server_result(self._h, ticket, ctypes.byref(rows), ctypes.byref(cols), ctypes.byref(lat)))
        return int(rows.value), int(cols.value), float(lat.value)

    def to_numpy(self, ticket: int, stream=None) -> np.ndarray:
        rows, cols, _ = self.result(ticket)
        out = np.empty((rows, cols), dtype=np.int32)
        if rows and cols:
            _check(_lib.gsmat_server_copy(self._h, ticket, out.ctypes.data, 0, _stream_ptr(stream)))
        return out

    def release(self, ticket: int):
        _check(_lib.gsmat_server_release(self._h, ticket))

    def stats(self) -> dict:
        s = ServerStats()
        _check(_lib.gsmat_server_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}


def batch_autotune(store: "Store", bgps, base: dict | None = None, stream=None) -> dict:
    arr, keep = _bgp_array(bgps)
    best = BatchConfig()
    cfg = _config(base)
    _check(_lib.gsmat_batch_autotune(store.handle, arr, len(bgps), ctypes.byref(cfg) if cfg else None,
                                     _stream_ptr(stream), ctypes.byref(best)))
    return {"block": best.block, "ctas_per_sm": best.ctas_per_sm, "arena_bytes": best.arena_bytes,
            "max_rows": best.max_rows, "use_graph": best.use_graph, "plan_cost": best.plan_cost,
            "expand_slots": best.expand_slots}


def plan(bgp, keys, stats, n_vars=None, cost: bool = False):
    """Host planner (Alg. 1; with ``cost``, the least-cost connected order of
    gsmat_plan_cost): (order, kinds, est) for given per-pattern keys and
    predicate statistics (list of dicts with nnz, nr_s, nr_o)."""
    pats, n, nv = _patterns(bgp)
    n_vars = nv if n_vars is None else n_vars
    k = np.ascontiguousarray(np.asarray(keys, dtype=np.int64))
    st = (PredStats * n)()
    for i, s in enumerate(stats):
        st[i] = PredStats(int(s.get("pred_id", 0)), int(s["nnz"]), int(s["nr_s"]), int(s["nr_o"]))
    order = np.zeros(n, np.int32)
    kinds = np.zeros(n, np.int32)
    est = np.zeros(n, np.float64)
    fn = _lib.gsmat_plan_cost if cost else _lib.gsmat_plan
    _check(fn(pats, n, int(n_vars), k.ctypes.data, st, order.ctypes.data, kinds.ctypes.data, est.ctypes.data))
    return order.tolist(), kinds.tolist(), est.tolist()


def _require(t, dtypes, n_min: int, what: str):
    """A contiguous CUDA tensor of one of `dtypes` with >= n_min elements: the
    library dereferences these pointers on the device, so a host tensor,
    a strided view or a short buffer is refused here."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{what}: a CUDA tensor is required")
    if t.dtype not in dtypes:
        raise ValueError(f"{what}: dtype {t.dtype} is not one of {tuple(dtypes)}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: the tensor must be contiguous")
    if t.numel() < n_min:
        raise ValueError(f"{what}: {t.numel()} elements, {n_min} needed")


def radix_sort_u64(keys, vals=None, begin_bit: int = 0, end_bit: int = 64, stream=None):
    """Sort a CUDA uint64/int64 tensor in place (optional int32/uint32 payload)."""
    import torch

    _require(keys, (torch.int64, torch.uint64), 0, "keys")
    if vals is not None:
        _require(vals, (torch.int32, torch.uint32), keys.numel(), "vals")
    _check(_lib.gsmat_radix_sort_u64(ctypes.c_void_p(keys.data_ptr()),
                                     ctypes.c_void_p(vals.data_ptr()) if vals is not None else None,
                                     keys.numel(), begin_bit, end_bit, _stream_ptr(stream)))


SORT_CARRY, SORT_GATHER = 1, 2


def sort_rows(cols, m: int, bits: int, out=None, stream=None, flags: int = 0):
    """Stable lexicographic reorder of the rows of V int32 CUDA columns by
    the first m; returns (or fills) V new columns.  flags: SORT_CARRY /
    SORT_GATHER force how the other columns travel (0: by size)."""
    import torch

    V = len(cols)
    n = cols[0].numel() if V else 0
    for i, c in enumerate(cols):
        _require(c, (torch.int32,), n, f"column {i}")
    if out is None:
        out = [c.new_empty(c.shape) for c in cols]
    if len(out) != V:
        raise ValueError(f"{len(out)} output columns for {V} input columns")
    for i, c in enumerate(out):
        _require(c, (torch.int32,), n, f"output column {i}")
    src = (ctypes.c_void_p * max(V, 1))(*[c.data_ptr() for c in cols])
    dst = (ctypes.c_void_p * max(V, 1))(*[c.data_ptr() for c in out])
    _check(_lib.gsmat_sort_rows(src, V, m, bits, n, dst, flags, _stream_ptr(stream)))
    return out


def exclusive_scan_i32(src, dst, stream=None):
    """dst[0..n] (int64 CUDA tensor) = exclusive prefix sums of src (int32)."""
    import torch

    _require(src, (torch.int32,), 0, "src")
    _require(dst, (torch.int64,), src.numel() + 1, "dst")
    _check(_lib.gsmat_exclusive_scan_i32(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                         src.numel(), _stream_ptr(stream)))


def exclusive_scan_i32_noalloc(src, dst, stream=None):
    """As exclusive_scan_i32, with no device allocation (static scratch;
    n <= exclusive_scan_i32_noalloc_max(); overlapping calls race)."""
    import torch

    _require(src, (torch.int32,), 0, "src")
    _require(dst, (torch.int64,), src.numel() + 1, "dst")
    _check(_lib.gsmat_exclusive_scan_i32_noalloc(ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                                 src.numel(), _stream_ptr(stream)))


def exclusive_scan_i32_noalloc_max() -> int:
    return int(_lib.gsmat_exclusive_scan_i32_noalloc_max())


def profile_enable(on: bool = True):
    _check(_lib.gsmat_profile_enable(1 if on else 0))


def launch_count() -> int:
    """Kernels the library has launched since it was loaded."""
    return int(_lib.gsmat_launch_count())


def profile_read(reset: bool = False) -> dict:
    n = ctypes.c_int32()
    _check(_lib.gsmat_profile_read(None, 0, ctypes.byref(n), 0))
    buf = (KernelProfile * max(1, n.value))()
    _check(_lib.gsmat_profile_read(buf, n.value, ctypes.byref(n), 1 if reset else 0))
    return {b.name.decode(): {"launches": b.launches, "total_ms": b.total_ms, "algo_bytes": b.algo_bytes,
                              "items": b.items} for b in buf[: n.value]}


# torch caching allocator as the device allocation hook -----------------------

_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_hooks = []


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch's caching
    allocator (enable=False restores cudaMallocAsync)."""
    if not enable:
        _check(_lib.gsmat_set_allocator(None, None, None))
        _hooks.clear()
        return
    import torch

    def _alloc(nbytes, ctx, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, ctx, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_T(_alloc), _FREE_T(_free)
    _hooks[:] = [a, f]
    _check(_lib.gsmat_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))
