"""ctypes binding of libsgm (include/sgm.h): the same entry points under the
same names, plus a small convenience wrapper (Engine) that marshals numpy
arrays and torch tensors. Every step of the matching runs inside libsgm's
kernels; this module only passes pointers and sizes and raises on errors.

There is no fallback: if libsgm.so cannot be built or loaded, import fails.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

# status codes (include/sgm.h)
SGM_OK = 0
SGM_W_TRUNCATED = 1
STATUS_NAMES = {
    0: "SGM_OK", 1: "SGM_W_TRUNCATED", -1: "SGM_E_INVALID_ARG", -2: "SGM_E_GRAPH_UNSORTED",
    -3: "SGM_E_GRAPH_SELF_LOOP", -4: "SGM_E_GRAPH_ASYMMETRIC", -5: "SGM_E_QUERY_DISCONNECTED",
    -6: "SGM_E_QUERY_TOO_LARGE", -7: "SGM_E_ORDER_NOT_CONNECTED", -8: "SGM_E_LABEL_RANGE", -9: "SGM_E_OOM",
    -10: "SGM_E_COUNT_OVERFLOW", -11: "SGM_E_DEVICE_TIMEOUT", -12: "SGM_E_QUEUE_OVERFLOW", -13: "SGM_E_TIME_CAP",
    -14: "SGM_E_CUDA", -15: "SGM_E_GRAPH_RANGE", -16: "SGM_E_QUERY_INVALID", -17: "SGM_E_WORK_CAP",
}
globals().update({v: k for k, v in STATUS_NAMES.items()})

SGM_HOST_PTRS = 0
SGM_DEVICE_PTRS = 1
SGM_BORROW = 2
SGM_VALIDATE = 4
SGM_MODE_COUNT = 0
SGM_MODE_HASH = 1
SGM_EXEC_FINE_BATCH = 0  # execution models of sgm_count (the ablation of Sec. 6.3)
SGM_EXEC_FINE_NAIVE = 1
SGM_EXEC_COARSE = 2

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64


class sgm_opts(ctypes.Structure):
    _fields_ = [("struct_size", _u32), ("mode", _i32), ("tau", _i64), ("pool_cap_bytes", _i64),
                ("use_filter", _i32), ("arith_last", _i32), ("warps_per_block", _i32), ("blocks_per_sm", _i32),
                ("split_min", _i32), ("sym_break", _i32), ("time_cap_s", ctypes.c_double),
                ("chunk_words", _i32), ("split_depth", _i32), ("pool_chunk", _i32), ("refine_rounds", _i32),
                ("work_cap", _u64), ("exec_model", _i32), ("unroll", _i32), ("steal_mode", _i32)]


class sgm_stats(ctypes.Structure):
    _fields_ = [("ms_filter", ctypes.c_double), ("ms_init", ctypes.c_double), ("ms_search", ctypes.c_double),
                ("init_depth", _i32), ("grid_blocks", _i32), ("pool_size", _i64), ("cand_checked", _u64),
                ("list_elems", _u64), ("search_probes", _u64), ("bitmap_probes", _u64), ("filter_probes", _u64),
                ("task_groups", _u64), ("steals", _u64), ("idle_lanes", _u64), ("scatter_rounds", _u64),
                ("launches", _u64), ("aut_size", _u64), ("alg_bytes", _u64), ("stack_bytes", _u64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


SGM_FEATURES = 32
SGM_MODEL_MAX_IN = 128


class sgm_graph_stats(ctypes.Structure):
    _fields_ = [("n", _i64), ("nnz", _i64), ("num_labels", _i32), ("reserved", _i32),
                ("label_frac", ctypes.c_double * 256), ("log2_deg_moment", ctypes.c_double * 4),
                ("deg_hist", ctypes.c_double * 8)]


class SgmError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().sgm_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_SIGS = {
    "sgm_opts_default": (None, [_vp]),
    "sgm_last_error": (ctypes.c_char_p, []),
    "sgm_create": (_i32, [_vp, _i32, _vp]),
    "sgm_set_stream": (_i32, [_vp, _vp]),
    "sgm_destroy": (_i32, [_vp]),
    "sgm_graph_load_csr": (_i32, [_vp, _i64, _vp, _vp, _vp, _i32, _u32, _vp]),
    "sgm_graph_free": (_i32, [_vp]),
    "sgm_graph_info": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "sgm_query_register": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
    "sgm_query_free": (_i32, [_vp]),
    "sgm_query_set_order": (_i32, [_vp, _vp, _i32]),
    "sgm_query_order_greedy": (_i32, [_vp, _vp]),
    "sgm_query_order_greedy_from": (_i32, [_vp, _vp, _i32]),
    "sgm_query_get_order": (_i32, [_vp, _vp]),
    "sgm_filter": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "sgm_refine": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _vp]),
    "sgm_cgraph_build": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp]),
    "sgm_cgraph_destroy": (_i32, [_vp]),
    "sgm_cgraph_edge_size": (_i32, [_vp, _i32, _i32, _vp, _vp]),
    "sgm_cgraph_edge_copy": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
    "sgm_count_cgraph": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "sgm_count": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sgm_count_root_range": (_i32, [_vp, _vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "sgm_enumerate": (_i32, [_vp, _vp, _vp, _vp, _vp, _u64, _vp, _vp, _vp]),
    "sgm_get_stats": (_i32, [_vp, _vp]),
    "sgm_query_automorphisms": (_i32, [_i32, _i32, _vp, _vp, _vp, _i32, _vp]),
    "sgm_query_greedy_order_host": (_i32, [_i32, _i32, _vp, _vp, _vp, _i32, _i32, _vp]),
    "sgm_query_symmetry_plan": (_i32, [_i32, _i32, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _i32, _vp, _vp]),
    "sgm_count_noalloc": (_i32, [_i32, _vp, _i64, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "sgm_batch_create": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _i32, _vp]),
    "sgm_batch_free": (_i32, [_vp]),
    "sgm_batch_run": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "sgm_batch_query_work": (_i32, [_vp, _vp]),
    "sgm_count_batch": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "sgm_graph_get_stats": (_i32, [_vp, _vp]),
    "sgm_features_from_stats": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp, _i64, _vp]),
    "sgm_prefix_features": (_i32, [_vp, _vp, _vp, _i64, _vp]),
    "sgm_model_create": (_i32, [_vp, _i32, _i32, _vp, _vp]),
    "sgm_model_free": (_i32, [_vp]),
    "sgm_model_info": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "sgm_model_get_params": (_i32, [_vp, _vp]),
    "sgm_model_set_params": (_i32, [_vp, _vp]),
    "sgm_model_forward": (_i32, [_vp, _vp, _i64, _vp]),
    "sgm_model_gradient": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "sgm_model_adam_step": (_i32, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "sgm_model_train": (_i32, [_vp, _vp, _vp, _i64, _i32, ctypes.c_float, _vp]),
    "sgm_query_order_learned": (_i32, [_vp, _vp, _vp, _i32, _i32, _i64, _vp, _vp, _vp]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libsgm.so, building it first with nvcc if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def _check(status, where):
    if status < 0:
        raise SgmError(status, where)
    return status


# ---------------------------------------------------------------------------
# the C entry points, one to one
# ---------------------------------------------------------------------------
def sgm_opts_default() -> sgm_opts:
    o = sgm_opts()
    lib().sgm_opts_default(ctypes.byref(o))
    return o


def sgm_last_error() -> str:
    return lib().sgm_last_error().decode(errors="replace")


def sgm_create(device: int = 0, stream: int | None = None):
    h = _vp()
    _check(lib().sgm_create(ctypes.byref(h), device, stream or None), "sgm_create")
    return h


def sgm_set_stream(e, stream):
    return _check(lib().sgm_set_stream(e, stream or None), "sgm_set_stream")


def sgm_destroy(e):
    return _check(lib().sgm_destroy(e), "sgm_destroy")


def sgm_graph_load_csr(e, n, rowptr_ptr, col_ptr, labels_ptr, num_labels, flags):
    h = _vp()
    _check(lib().sgm_graph_load_csr(e, n, rowptr_ptr, col_ptr, labels_ptr, num_labels, flags, ctypes.byref(h)),
           "sgm_graph_load_csr")
    return h


def sgm_graph_free(g):
    return _check(lib().sgm_graph_free(g), "sgm_graph_free")


def sgm_graph_info(g):
    n, nnz, dmax, hubs = _i64(), _i64(), _i32(), _i32()
    _check(lib().sgm_graph_info(g, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(dmax), ctypes.byref(hubs)),
           "sgm_graph_info")
    return dict(n=n.value, nnz=nnz.value, dmax=dmax.value, hubs=hubs.value)


def sgm_query_register(e, k, edges, labels=None):
    ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    lb = None if labels is None else np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    h = _vp()
    _check(lib().sgm_query_register(e, k, len(ed) // 2, ed.ctypes.data_as(_vp),
                                     None if lb is None else lb.ctypes.data_as(_vp), ctypes.byref(h)),
           "sgm_query_register")
    return h


def sgm_query_free(q):
    return _check(lib().sgm_query_free(q), "sgm_query_free")


def sgm_query_set_order(q, phi):
    p = np.ascontiguousarray(np.asarray(phi, dtype=np.int32))
    return _check(lib().sgm_query_set_order(q, p.ctypes.data_as(_vp), len(p)), "sgm_query_set_order")


def sgm_query_order_greedy(q, g):
    return _check(lib().sgm_query_order_greedy(q, g), "sgm_query_order_greedy")


def sgm_query_order_greedy_from(q, g, root):
    return _check(lib().sgm_query_order_greedy_from(q, g, root), "sgm_query_order_greedy_from")


def sgm_query_get_order(q, k):
    out = np.zeros(k, dtype=np.int32)
    _check(lib().sgm_query_get_order(q, out.ctypes.data_as(_vp)), "sgm_query_get_order")
    return out


def sgm_filter(e, g, q, use_filter, dev_bits_ptr):
    return _check(lib().sgm_filter(e, g, q, use_filter, dev_bits_ptr), "sgm_filter")


def sgm_refine(e, g, q, use_filter, max_rounds, dev_bits_ptr) -> int:
    rounds = _i32()
    _check(lib().sgm_refine(e, g, q, use_filter, max_rounds, dev_bits_ptr, ctypes.byref(rounds)), "sgm_refine")
    return rounds.value


def sgm_cgraph_build(e, g, q, use_filter=1, refine_rounds=0):
    h = _vp()
    _check(lib().sgm_cgraph_build(e, g, q, use_filter, refine_rounds, ctypes.byref(h)), "sgm_cgraph_build")
    return h


def sgm_cgraph_destroy(c):
    _check(lib().sgm_cgraph_destroy(c), "sgm_cgraph_destroy")


def sgm_cgraph_edge(c, u, u2):
    """Directed edge (u, u2) of G' as host arrays: (vs int32, ptr int64, adj int32)."""
    rows, entries = _i64(), _i64()
    _check(lib().sgm_cgraph_edge_size(c, u, u2, ctypes.byref(rows), ctypes.byref(entries)), "sgm_cgraph_edge_size")
    vs = np.zeros(rows.value, dtype=np.int32)
    ptr = np.zeros(rows.value + 1, dtype=np.int64)
    adj = np.zeros(entries.value, dtype=np.int32)
    _check(lib().sgm_cgraph_edge_copy(c, u, u2, vs.ctypes.data_as(_vp), ptr.ctypes.data_as(_vp),
                                      adj.ctypes.data_as(_vp)), "sgm_cgraph_edge_copy")
    return vs, ptr, adj


def sgm_count_cgraph(e, g, q, c, opts=None, want_hash=False, k=None, root_range=(0, 1 << 62)):
    cnt, h = _u64(), _u64()
    lv = np.zeros(32, dtype=np.uint64)
    _check(lib().sgm_count_cgraph(e, g, q, c, None if opts is None else ctypes.byref(opts), int(root_range[0]),
                                  int(root_range[1]), ctypes.byref(cnt),
                                  ctypes.byref(h) if want_hash else None, lv.ctypes.data_as(_vp)),
           "sgm_count_cgraph")
    return dict(count=cnt.value, hash=h.value if want_hash else None, level_counts=lv[:k] if k else lv)


def sgm_count(e, g, q, opts=None, want_hash=False, k=None):
    c, h = _u64(), _u64()
    lv = np.zeros(32, dtype=np.uint64)
    _check(lib().sgm_count(e, g, q, None if opts is None else ctypes.byref(opts), ctypes.byref(c),
                           ctypes.byref(h) if want_hash else None, lv.ctypes.data_as(_vp)), "sgm_count")
    return dict(count=c.value, hash=h.value if want_hash else None, level_counts=lv[:k] if k else lv)


def sgm_count_root_range(e, g, q, lo, hi, opts=None, want_hash=False, k=None):
    c, h = _u64(), _u64()
    lv = np.zeros(32, dtype=np.uint64)
    _check(lib().sgm_count_root_range(e, g, q, None if opts is None else ctypes.byref(opts), lo, hi, ctypes.byref(c),
                                      ctypes.byref(h) if want_hash else None, lv.ctypes.data_as(_vp)),
           "sgm_count_root_range")
    return dict(count=c.value, hash=h.value if want_hash else None, level_counts=lv[:k] if k else lv)


def sgm_enumerate(e, g, q, dev_out_ptr, cap, opts=None):
    w, t, h = _u64(), _u64(), _u64()
    st = _check(lib().sgm_enumerate(e, g, q, None if opts is None else ctypes.byref(opts), dev_out_ptr, cap,
                                    ctypes.byref(w), ctypes.byref(t), ctypes.byref(h)), "sgm_enumerate")
    return dict(written=w.value, total=t.value, hash=h.value, truncated=st == SGM_W_TRUNCATED)


def sgm_query_automorphisms(k, edges, labels=None, cap=4096) -> np.ndarray:
    ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    lb = None if labels is None else np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    out = np.zeros((cap, k), dtype=np.int32)
    n = _i32()
    _check(lib().sgm_query_automorphisms(k, len(ed) // 2, ed.ctypes.data_as(_vp),
                                         None if lb is None else lb.ctypes.data_as(_vp), out.ctypes.data_as(_vp),
                                         cap, ctypes.byref(n)), "sgm_query_automorphisms")
    return out[:min(n.value, cap)]


def sgm_query_greedy_order_host(k, edges, labels=None, label_count=None, root=-1) -> np.ndarray:
    ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    lb = None if labels is None else np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    lc = np.ascontiguousarray(np.asarray([] if label_count is None else label_count, dtype=np.uint64))
    out = np.zeros(k, dtype=np.int32)
    _check(lib().sgm_query_greedy_order_host(k, len(ed) // 2, ed.ctypes.data_as(_vp),
                                             None if lb is None else lb.ctypes.data_as(_vp),
                                             lc.ctypes.data_as(_vp) if len(lc) else None, len(lc), root,
                                             out.ctypes.data_as(_vp)), "sgm_query_greedy_order_host")
    return out


def sgm_query_symmetry_plan(k, edges, labels, phi, count_mode=False, group_cap=4096) -> dict:
    ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    lb = None if labels is None else np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    ph = np.ascontiguousarray(np.asarray(phi, dtype=np.int32))
    gt = np.zeros(k, dtype=np.uint32)
    up = np.zeros(k, dtype=np.uint32)
    grp = np.zeros((group_cap, k), dtype=np.int32)
    n, ar = _i32(), _i32()
    _check(lib().sgm_query_symmetry_plan(k, len(ed) // 2, ed.ctypes.data_as(_vp),
                                         None if lb is None else lb.ctypes.data_as(_vp), ph.ctypes.data_as(_vp),
                                         1 if count_mode else 0, gt.ctypes.data_as(_vp), up.ctypes.data_as(_vp),
                                         grp.ctypes.data_as(_vp), group_cap, ctypes.byref(n), ctypes.byref(ar)),
           "sgm_query_symmetry_plan")
    return dict(sb_gt=gt, up=up, group=grp[:min(n.value, group_cap)], group_n=n.value, arith=bool(ar.value))


def sgm_get_stats(e) -> dict:
    s = sgm_stats()
    _check(lib().sgm_get_stats(e, ctypes.byref(s)), "sgm_get_stats")
    return s.as_dict()


def sgm_count_noalloc(device, stream, n, rowptr_ptr, col_ptr, labels_ptr, num_labels, k, edges, labels=None,
                      phi=None):
    """Count with no allocation inside libsgm; graph arrays are device pointers."""
    ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    lb = None if labels is None else np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    ph = None if phi is None else np.ascontiguousarray(np.asarray(phi, dtype=np.int32))
    c = _u64()
    _check(lib().sgm_count_noalloc(device, stream or None, n, rowptr_ptr, col_ptr, labels_ptr, num_labels, k,
                                   len(ed) // 2, ed.ctypes.data_as(_vp),
                                   None if lb is None else lb.ctypes.data_as(_vp),
                                   None if ph is None else ph.ctypes.data_as(_vp), ctypes.byref(c)),
           "sgm_count_noalloc")
    return c.value


def _handles(qs):
    arr = (_vp * max(1, len(qs)))()
    for i, q in enumerate(qs):
        arr[i] = q
    return arr


def _ranges(root_ranges, nq):
    if root_ranges is None:
        return None, None
    r = np.ascontiguousarray(np.asarray(root_ranges, dtype=np.int64).reshape(nq, 2))
    return r, r.ctypes.data_as(_vp)


def sgm_batch_create(e, g, qs, opts=None, want_hash=False, root_ranges=None):
    h = _vp()
    keep, rp = _ranges(root_ranges, len(qs))
    _check(lib().sgm_batch_create(e, g, _handles(qs), len(qs), rp, None if opts is None else ctypes.byref(opts),
                                  1 if want_hash else 0, ctypes.byref(h)), "sgm_batch_create")
    del keep
    return h


def sgm_batch_free(b):
    return _check(lib().sgm_batch_free(b), "sgm_batch_free")


def sgm_batch_run(b, nq, want_hash=False, check=True):
    counts = np.zeros(max(nq, 1), dtype=np.uint64)
    hashes = np.zeros(max(nq, 1), dtype=np.uint64)
    statuses = np.zeros(max(nq, 1), dtype=np.int32)
    ms = ctypes.c_double()
    st = lib().sgm_batch_run(b, counts.ctypes.data_as(_vp), hashes.ctypes.data_as(_vp) if want_hash else None,
                             statuses.ctypes.data_as(_vp), ctypes.byref(ms))
    if check:
        _check(st, "sgm_batch_run")
    return dict(counts=counts[:nq], hashes=hashes[:nq] if want_hash else None, statuses=statuses[:nq],
                ms=ms.value, status=st)


def sgm_batch_query_work(b, nq):
    work = np.zeros(max(nq, 1), dtype=np.uint64)
    _check(lib().sgm_batch_query_work(b, work.ctypes.data_as(_vp)), "sgm_batch_query_work")
    return work[:nq]


def sgm_count_batch(e, g, qs, opts=None, want_hash=False, root_ranges=None):
    nq = len(qs)
    counts = np.zeros(max(nq, 1), dtype=np.uint64)
    hashes = np.zeros(max(nq, 1), dtype=np.uint64)
    statuses = np.zeros(max(nq, 1), dtype=np.int32)
    keep, rp = _ranges(root_ranges, nq)
    _check(lib().sgm_count_batch(e, g, _handles(qs), nq, rp, None if opts is None else ctypes.byref(opts),
                                 counts.ctypes.data_as(_vp), hashes.ctypes.data_as(_vp) if want_hash else None,
                                 statuses.ctypes.data_as(_vp)), "sgm_count_batch")
    return dict(counts=counts[:nq], hashes=hashes[:nq] if want_hash else None, statuses=statuses[:nq])


def sgm_graph_get_stats(g) -> sgm_graph_stats:
    st = sgm_graph_stats()
    _check(lib().sgm_graph_get_stats(g, ctypes.byref(st)), "sgm_graph_get_stats")
    return st


def sgm_features_from_stats(stats: sgm_graph_stats, k, edges, labels, phi, anchor_deg=-1) -> np.ndarray:
    ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    lb = None if labels is None else np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    ph = np.ascontiguousarray(np.asarray(phi, dtype=np.int32))
    out = np.zeros((k, SGM_FEATURES), dtype=np.float32)
    _check(lib().sgm_features_from_stats(ctypes.byref(stats), k, len(ed) // 2, ed.ctypes.data_as(_vp),
                                         None if lb is None else lb.ctypes.data_as(_vp), ph.ctypes.data_as(_vp),
                                         anchor_deg, out.ctypes.data_as(_vp)), "sgm_features_from_stats")
    return out


def sgm_prefix_features(q, g, k, phi=None, anchor=-1) -> np.ndarray:
    ph = None if phi is None else np.ascontiguousarray(np.asarray(phi, dtype=np.int32))
    out = np.zeros((k, SGM_FEATURES), dtype=np.float32)
    _check(lib().sgm_prefix_features(q, g, None if ph is None else ph.ctypes.data_as(_vp), anchor,
                                     out.ctypes.data_as(_vp)), "sgm_prefix_features")
    return out


def sgm_model_create(e, in_dim, hidden, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    h = _vp()
    _check(lib().sgm_model_create(e, in_dim, hidden, p.ctypes.data_as(_vp), ctypes.byref(h)), "sgm_model_create")
    return h


def sgm_model_free(m):
    return _check(lib().sgm_model_free(m), "sgm_model_free")


def sgm_model_info(m) -> dict:
    a, b, c, d = _i32(), _i32(), _i64(), _i64()
    _check(lib().sgm_model_info(m, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)),
           "sgm_model_info")
    return dict(in_dim=a.value, hidden=b.value, n_params=c.value, steps=d.value)


def sgm_model_get_params(m, n_params) -> np.ndarray:
    out = np.zeros(n_params, dtype=np.float32)
    _check(lib().sgm_model_get_params(m, out.ctypes.data_as(_vp)), "sgm_model_get_params")
    return out


def sgm_model_set_params(m, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    return _check(lib().sgm_model_set_params(m, p.ctypes.data_as(_vp)), "sgm_model_set_params")


def sgm_model_forward(m, X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.zeros(len(X), dtype=np.float32)
    _check(lib().sgm_model_forward(m, X.ctypes.data_as(_vp), len(X), y.ctypes.data_as(_vp)), "sgm_model_forward")
    return y


def sgm_model_gradient(m, X, t, n_params):
    X = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    g = np.zeros(n_params, dtype=np.float32)
    loss = ctypes.c_float()
    _check(lib().sgm_model_gradient(m, X.ctypes.data_as(_vp), t.ctypes.data_as(_vp), len(X), g.ctypes.data_as(_vp),
                                    ctypes.byref(loss)), "sgm_model_gradient")
    return g, float(loss.value)


def sgm_model_adam_step(m, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    return _check(lib().sgm_model_adam_step(m, lr, beta1, beta2, eps), "sgm_model_adam_step")


def sgm_model_train(m, X, t, steps, lr) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    losses = np.zeros(max(steps, 1), dtype=np.float32)
    _check(lib().sgm_model_train(m, X.ctypes.data_as(_vp), t.ctypes.data_as(_vp), len(X), steps, lr,
                                 losses.ctypes.data_as(_vp)), "sgm_model_train")
    return losses[:steps]


def sgm_query_order_learned(q, g, m, beam=8, root=-1, anchor=-1) -> dict:
    pl, pg, used = ctypes.c_double(), ctypes.c_double(), _i32()
    _check(lib().sgm_query_order_learned(q, g, m, beam, root, anchor, ctypes.byref(pl), ctypes.byref(pg),
                                         ctypes.byref(used)), "sgm_query_order_learned")
    return dict(pred_learned=pl.value, pred_greedy=pg.value, used_learned=bool(used.value))


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
def _host_ptr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_vp)


class Graph:
    def __init__(self, engine, handle, keep):
        self.engine = engine
        self.handle = handle
        self._keep = keep
        self.info = sgm_graph_info(handle)

    def stats(self) -> sgm_graph_stats:
        return sgm_graph_get_stats(self.handle)

    def free(self):
        if self.handle:
            sgm_graph_free(self.handle)
            self.handle = None


class Query:
    def __init__(self, engine, handle, k):
        self.engine = engine
        self.handle = handle
        self.k = k

    def set_order(self, phi):
        sgm_query_set_order(self.handle, phi)

    def order_greedy(self, graph, root=None):
        if root is None:
            sgm_query_order_greedy(self.handle, graph.handle)
        else:
            sgm_query_order_greedy_from(self.handle, graph.handle, root)

    def order(self):
        return sgm_query_get_order(self.handle, self.k)

    def features(self, graph, phi=None, anchor=-1):
        return sgm_prefix_features(self.handle, graph.handle, self.k, phi, anchor)

    def order_learned(self, graph, model, beam=8, root=-1, anchor=-1):
        return sgm_query_order_learned(self.handle, graph.handle, model.handle, beam, root, anchor)

    def free(self):
        if self.handle:
            sgm_query_free(self.handle)
            self.handle = None


class Model:
    """The cost-model MLP on the engine's device (see sgm_model_create)."""

    def __init__(self, engine, in_dim, hidden, params):
        self.engine = engine
        self.handle = sgm_model_create(engine.handle, in_dim, hidden, params)
        self.info = sgm_model_info(self.handle)

    def params(self):
        return sgm_model_get_params(self.handle, self.info["n_params"])

    def set_params(self, p):
        sgm_model_set_params(self.handle, p)

    def forward(self, X):
        return sgm_model_forward(self.handle, X)

    def gradient(self, X, t):
        return sgm_model_gradient(self.handle, X, t, self.info["n_params"])

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        sgm_model_adam_step(self.handle, lr, beta1, beta2, eps)

    def train(self, X, t, steps, lr):
        return sgm_model_train(self.handle, X, t, steps, lr)

    def free(self):
        if self.handle:
            sgm_model_free(self.handle)
            self.handle = None


class CandidateGraph:
    """The candidate graph G' of one query on the device (sgm_cgraph_build)."""

    def __init__(self, engine, graph, query, use_filter=True, refine_rounds=0):
        self.engine = engine
        self.graph = graph
        self.query = query
        self.handle = sgm_cgraph_build(engine.handle, graph.handle, query.handle, 1 if use_filter else 0,
                                       refine_rounds)

    def edge(self, u, u2):
        """(vs, ptr, adj): the vertices of C(u) ascending and, per vertex, the
        sorted list N(v) ∩ C(u2) as adj[ptr[i]:ptr[i+1]]."""
        return sgm_cgraph_edge(self.handle, u, u2)

    def count(self, want_hash=False, root_range=None, **opts) -> dict:
        r = sgm_count_cgraph(self.engine.handle, self.graph.handle, self.query.handle, self.handle,
                             self.engine.opts(**opts), want_hash, self.query.k,
                             (0, self.graph.info["n"]) if root_range is None else root_range)
        r["stats"] = sgm_get_stats(self.engine.handle)
        return r

    def free(self):
        if self.handle:
            sgm_cgraph_destroy(self.handle)
            self.handle = None


class Batch:
    """Many queries in one captured persistent launch (see sgm_batch_create)."""

    def __init__(self, engine, graph, queries, want_hash=False, root_ranges=None, **opts):
        self.engine = engine
        self.nq = len(queries)
        self.want_hash = want_hash
        self.handle = sgm_batch_create(engine.handle, graph.handle, [q.handle for q in queries],
                                       engine.opts(**opts), want_hash, root_ranges)

    def run(self, check=True) -> dict:
        r = sgm_batch_run(self.handle, self.nq, self.want_hash, check)
        r["stats"] = sgm_get_stats(self.engine.handle)
        r["work"] = sgm_batch_query_work(self.handle, self.nq)
        return r

    def free(self):
        if self.handle:
            sgm_batch_free(self.handle)
            self.handle = None


class Engine:
    """One engine on one CUDA device. Graph arrays may be numpy (host) or torch
    CUDA tensors (device); outputs of enumerate go into a torch CUDA tensor."""

    def __init__(self, device: int = 0, stream=None):
        self.device = device
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = None
        self.handle = sgm_create(device, stream)

    def close(self):
        if self.handle:
            sgm_destroy(self.handle)
            self.handle = None

    def load_graph(self, rowptr, col, labels=None, num_labels=1, validate=True, borrow=False) -> Graph:
        flags = SGM_VALIDATE if validate else 0
        keep = []
        if hasattr(rowptr, "is_cuda") and rowptr.is_cuda:
            flags |= SGM_DEVICE_PTRS | (SGM_BORROW if borrow else 0)
            n = rowptr.numel() - 1
            rp, cp = rowptr.data_ptr(), col.data_ptr()
            lp = labels.data_ptr() if labels is not None else None
            keep = [rowptr, col, labels]
        else:
            n = len(rowptr) - 1
            r, rp = _host_ptr(rowptr, np.int64)
            c, cp = _host_ptr(col, np.int32)
            keep = [r, c]
            lp = None
            if labels is not None:
                l, lp = _host_ptr(labels, np.int32)
                keep.append(l)
        h = sgm_graph_load_csr(self.handle, n, rp, cp, lp, num_labels if labels is not None else 1, flags)
        return Graph(self, h, keep if borrow else None)

    def batch(self, graph, queries, want_hash=False, root_ranges=None, **opts) -> Batch:
        return Batch(self, graph, queries, want_hash, root_ranges, **opts)

    def count_batch(self, graph, queries, want_hash=False, root_ranges=None, **opts) -> dict:
        return sgm_count_batch(self.handle, graph.handle, [q.handle for q in queries], self.opts(**opts), want_hash,
                               root_ranges)

    def model(self, in_dim, hidden, params) -> Model:
        return Model(self, in_dim, hidden, params)

    def query(self, k, edges, labels=None) -> Query:
        return Query(self, sgm_query_register(self.handle, k, edges, labels), k)

    def opts(self, **kw) -> sgm_opts:
        o = sgm_opts_default()
        fields = {f for f, _ in sgm_opts._fields_}
        for key, val in kw.items():
            if key not in fields or key == "struct_size":
                raise TypeError(f"unknown sgm_opts field {key!r}")
            setattr(o, key, val)
        return o

    def count(self, graph: Graph, query: Query, want_hash=False, root_range=None, **opts) -> dict:
        o = self.opts(**opts)
        if root_range is None:
            r = sgm_count(self.handle, graph.handle, query.handle, o, want_hash, query.k)
        else:
            r = sgm_count_root_range(self.handle, graph.handle, query.handle, root_range[0], root_range[1], o,
                                     want_hash, query.k)
        r["stats"] = sgm_get_stats(self.handle)
        return r

    def enumerate(self, graph: Graph, query: Query, cap: int, **opts):
        import torch
        out = torch.empty((max(cap, 1), query.k), dtype=torch.int32, device=f"cuda:{self.device}")
        r = sgm_enumerate(self.handle, graph.handle, query.handle, out.data_ptr(), cap, self.opts(**opts))
        r["rows"] = out[:r["written"]]
        r["stats"] = sgm_get_stats(self.handle)
        return r

    def candidate_graph(self, graph: Graph, query: Query, use_filter=True, refine_rounds=0) -> "CandidateGraph":
        return CandidateGraph(self, graph, query, use_filter, refine_rounds)

    def filter_bits(self, graph: Graph, query: Query, use_filter=True):
        import torch
        words = (graph.info["n"] + 31) // 32
        out = torch.zeros((query.k, max(words, 1)), dtype=torch.int32, device=f"cuda:{self.device}")
        sgm_filter(self.handle, graph.handle, query.handle, 1 if use_filter else 0, out.data_ptr())
        return out

    def refine_bits(self, graph: Graph, query: Query, max_rounds: int, use_filter=True):
        """(refined candidate bitmaps [k, words] int32 on the device, rounds that cleared a candidate)."""
        import torch
        words = (graph.info["n"] + 31) // 32
        out = torch.zeros((query.k, max(words, 1)), dtype=torch.int32, device=f"cuda:{self.device}")
        rounds = sgm_refine(self.handle, graph.handle, query.handle, 1 if use_filter else 0, max_rounds,
                            out.data_ptr())
        return out, rounds
