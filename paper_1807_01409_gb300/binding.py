"""Thin Python binding of libtid.so (include/tid.h), by ctypes.

The functions carry the C names and only marshal arguments: every step of the
query path runs in the library's CUDA kernels.  Device buffers may be torch
CUDA tensors (their ``data_ptr()`` is passed); host buffers numpy arrays.  If the
library has not been built, the first call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtid.so")

TID_OK, TID_ERR_ARG, TID_ERR_ID, TID_ERR_OOM, TID_ERR_CAPACITY, TID_ERR_TIMEOUT, TID_ERR_CUDA = range(7)
TID_HOST, TID_DEVICE = 0, 1
TID_MAX_COLS = 8
TID_MAX_MULTI = 16
TID_BATCH_KEYS = 1920
ERR_NAMES = {0: "TID_OK", 1: "TID_ERR_ARG", 2: "TID_ERR_ID", 3: "TID_ERR_OOM",
             4: "TID_ERR_CAPACITY", 5: "TID_ERR_TIMEOUT", 6: "TID_ERR_CUDA"}


class TidError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class tid_pattern(C.Structure):
    _fields_ = [("s", C.c_int32), ("p", C.c_int32), ("o", C.c_int32),
                ("var", C.c_int8 * 3), ("reserved", C.c_int8)]


class tid_server_config(C.Structure):
    _fields_ = [("workers", C.c_int32), ("max_wave", C.c_int32), ("batch_scans", C.c_int32),
                ("reserved", C.c_int32), ("budget_bytes", C.c_int64)]


class tid_server_stats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("submitted", "completed", "failed", "waves", "max_wave_seen",
                                         "peak_admitted_bytes", "scan_patterns", "budget_waits")]


TID_REQ_INDEX, TID_REQ_PLAN = 1, 2


class tid_rdfs_vocab(C.Structure):
    _fields_ = [("type", C.c_int32), ("domain", C.c_int32), ("range", C.c_int32),
                ("sub_property_of", C.c_int32), ("sub_class_of", C.c_int32)]


class tid_entail_stats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("res1", "dist1", "res2", "dist2", "all")]


RULES = (2, 3, 5, 7, 9, 11)


class tid_pred(C.Structure):
    _fields_ = [("var", C.c_int32), ("op", C.c_int32), ("a", C.c_int32), ("b", C.c_int32)]


class tid_plan_node(C.Structure):
    _fields_ = [("op", C.c_int32), ("n_in", C.c_int32), ("in_", C.c_int32 * 4),
                ("pattern", tid_pattern), ("pred", tid_pred), ("algo", C.c_int32),
                ("n_vars", C.c_int32), ("vars", C.c_int8 * 8)]


CMP = {"eq": 0, "ne": 1, "lt": 2, "le": 3, "gt": 4, "ge": 5, "range": 6}
TID_JOIN_LEFT, TID_JOIN_RIGHT = 0x100, 0x200
TID_JOIN_FULL = TID_JOIN_LEFT | TID_JOIN_RIGHT
JOIN = {"auto": 0, "sort_merge": 1, "sortmerge": 1, "hash": 2, "left": TID_JOIN_LEFT, "right": TID_JOIN_RIGHT,
        "full": TID_JOIN_FULL}
OP = {"match": 1, "filter": 2, "join": 3, "union": 4, "project": 5}


def make_pattern(s=0, p=0, o=0, var=(-1, -1, -1)) -> tid_pattern:
    """A pattern from (s, p, o) with 0 = "?", and variable ids per slot (-1 = none)."""
    pt = tid_pattern()
    pt.s, pt.p, pt.o = int(s), int(p), int(o)
    for j in range(3):
        pt.var[j] = int(var[j])
    pt.reserved = 0
    return pt


def as_pattern(x) -> tid_pattern:
    if isinstance(x, tid_pattern):
        return x
    if hasattr(x, "key") and hasattr(x, "var"):
        return make_pattern(*x.key(), var=x.var)
    x = tuple(x)
    return make_pattern(*x[:3], var=x[3] if len(x) > 3 else (-1, -1, -1))


_lib = None
_vp = C.c_void_p


def lib():
    """Load libtid.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libtid.so not built ({LIB_PATH}); run paper_1807_01409_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    i32p, i64p, i8p = C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int8)
    sig = {
        "tid_last_error": (C.c_char_p, []),
        "tid_ctx_create": (C.c_int, [C.c_int, _vp, C.POINTER(_vp)]),
        "tid_ctx_sync": (C.c_int, [_vp]),
        "tid_ctx_destroy": (C.c_int, [_vp]),
        "tid_load": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int64, C.c_int, C.c_int, C.POINTER(_vp)]),
        "tid_store_info": (C.c_int, [_vp, i64p, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp)]),
        "tid_store_free": (C.c_int, [_vp]),
        "tid_match": (C.c_int, [_vp, _vp, tid_pattern, C.POINTER(_vp)]),
        "tid_set_rows": (C.c_int, [_vp, i64p]),
        "tid_set_info": (C.c_int, [_vp, C.POINTER(C.c_int), i64p, C.POINTER(i8p),
                                   C.POINTER(C.POINTER(_vp)), C.POINTER(_vp)]),
        "tid_set_to_host": (C.c_int, [_vp, _vp, C.c_int64, i64p]),
        "tid_set_free": (C.c_int, [_vp]),
        "tid_match_multi": (C.c_int, [_vp, _vp, C.POINTER(tid_pattern), C.c_int, C.POINTER(_vp)]),
        "tid_match_batch": (C.c_int, [_vp, _vp, C.POINTER(tid_pattern), C.c_int, C.POINTER(_vp)]),
        "tid_bind": (C.c_int, [_vp, _vp, tid_pattern, _vp, C.POINTER(tid_pred), C.c_int, C.POINTER(_vp)]),
        "tid_filter": (C.c_int, [_vp, _vp, C.POINTER(tid_pred), C.c_int, C.POINTER(_vp)]),
        "tid_join": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(_vp)]),
        "tid_union": (C.c_int, [_vp, C.POINTER(_vp), C.c_int, C.POINTER(_vp)]),
        "tid_project": (C.c_int, [_vp, _vp, C.POINTER(C.c_int8), C.c_int, C.POINTER(_vp)]),
        "tid_set_from_host": (C.c_int, [_vp, _vp, C.c_int64, C.c_int, C.POINTER(C.c_int8), C.POINTER(_vp)]),
        "tid_exec": (C.c_int, [_vp, _vp, C.POINTER(tid_plan_node), C.c_int, C.POINTER(_vp)]),
        "tid_plan_check": (C.c_int, [C.POINTER(tid_plan_node), C.c_int]),
        "tid_batch_tuning": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "tid_batch_table_check": (C.c_int, [C.POINTER(tid_pattern), C.c_int, C.c_uint32, C.POINTER(C.c_int),
                                            C.POINTER(C.c_int)]),
        "tid_match_noalloc": (C.c_int, [C.c_int, _vp, _vp, _vp, _vp, C.c_int64, tid_pattern, _vp, C.c_int64,
                                        _vp]),
        "tid_ctx_inject_alloc_failure": (C.c_int, [_vp, C.c_int64]),
        "tid_ctx_test_bounded_wait": (C.c_int, [_vp, C.c_int64]),
        "tid_entail": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(tid_rdfs_vocab), C.POINTER(_vp),
                                 C.POINTER(tid_entail_stats)]),
        "tid_server_create": (C.c_int, [C.c_int, _vp, _vp, _vp, C.c_int64, C.POINTER(tid_server_config),
                                        C.POINTER(_vp)]),
        "tid_server_now_ns": (C.c_int64, []),
        "tid_server_submit": (C.c_int, [_vp, C.c_int, C.POINTER(tid_plan_node), C.c_int, C.c_int64, i64p]),
        "tid_server_wait": (C.c_int, [_vp, C.c_int64, C.c_int64]),
        "tid_server_result": (C.c_int, [_vp, C.c_int64, C.POINTER(C.c_int), C.POINTER(C.c_int), i8p, i64p,
                                        C.POINTER(i32p), i64p]),
        "tid_server_release": (C.c_int, [_vp, C.c_int64]),
        "tid_server_get_stats": (C.c_int, [_vp, C.POINTER(tid_server_stats)]),
        "tid_server_destroy": (C.c_int, [_vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    return lib().tid_last_error().decode()


def _rows(x):
    """Length of an array or tensor argument, None for a raw address."""
    return int(x.shape[0]) if hasattr(x, "shape") and len(x.shape) > 0 else None


def _int_dtype(x, name, bits):
    if hasattr(x, "dtype") and str(x.dtype) not in (f"int{bits}", f"torch.int{bits}"):
        raise TypeError(f"{name} must be int{bits}")


def _within(n, name, *arrays):
    """n elements must fit every array argument (the library trusts the sizes)."""
    for a in arrays:
        L = _rows(a)
        if L is not None and n > L:
            raise ValueError(f"{name} = {n} exceeds an argument of length {L}")


def _check(rc, what):
    if rc != TID_OK:
        raise TidError(rc, f"{what}: {last_error()}")


def _ptr(x):
    """Address of a torch tensor / numpy array / int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


# ---------------------------------------------------------------------------
# C entry points (same names)
# ---------------------------------------------------------------------------

def tid_ctx_create(device: int = 0, stream=None):
    """stream: a cudaStream_t as int (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    out = _vp()
    _check(lib().tid_ctx_create(int(device), stream if stream else None, C.byref(out)), "tid_ctx_create")
    return out


def tid_ctx_sync(ctx):
    _check(lib().tid_ctx_sync(ctx), "tid_ctx_sync")


def tid_ctx_destroy(ctx):
    _check(lib().tid_ctx_destroy(ctx), "tid_ctx_destroy")


def tid_load(ctx, s, p, o, n=None, where=None, copy=1):
    """Columns are torch CUDA tensors (where=TID_DEVICE), or numpy / CPU tensors (TID_HOST)."""
    if n is None:
        n = int(s.shape[0])
    if where is None:
        where = TID_DEVICE if (hasattr(s, "is_cuda") and s.is_cuda) else TID_HOST
    for c in (s, p, o):
        if hasattr(c, "dtype") and str(c.dtype) not in ("int32", "torch.int32"):
            raise TypeError("store columns must be int32")
        if isinstance(c, np.ndarray) and not c.flags["C_CONTIGUOUS"]:
            raise ValueError("store columns must be contiguous")
        if hasattr(c, "is_contiguous") and not c.is_contiguous():
            raise ValueError("store columns must be contiguous")
    _within(int(n), "n", s, p, o)
    out = _vp()
    _check(lib().tid_load(ctx, _ptr(s), _ptr(p), _ptr(o), int(n), int(where), int(copy), C.byref(out)),
           "tid_load")
    return out


def tid_store_info(st):
    n = C.c_int64()
    s, p, o = _vp(), _vp(), _vp()
    _check(lib().tid_store_info(st, C.byref(n), C.byref(s), C.byref(p), C.byref(o)), "tid_store_info")
    return n.value, s.value, p.value, o.value


def tid_store_free(st):
    _check(lib().tid_store_free(st), "tid_store_free")


def tid_match(ctx, st, pattern):
    out = _vp()
    _check(lib().tid_match(ctx, st, as_pattern(pattern), C.byref(out)), "tid_match")
    return out


def tid_set_rows(set_) -> int:
    r = C.c_int64()
    _check(lib().tid_set_rows(set_, C.byref(r)), "tid_set_rows")
    return r.value


def tid_set_info(set_):
    k = C.c_int()
    cap = C.c_int64()
    vars_ = C.POINTER(C.c_int8)()
    cols = C.POINTER(_vp)()
    drows = _vp()
    _check(lib().tid_set_info(set_, C.byref(k), C.byref(cap), C.byref(vars_), C.byref(cols),
                              C.byref(drows)), "tid_set_info")
    return {"cols": k.value, "capacity": cap.value,
            "vars": tuple(vars_[i] for i in range(k.value)),
            "dev_cols": tuple(cols[i] for i in range(k.value)), "dev_rows": drows.value}


def tid_set_to_host(set_, buf=None):
    """Rows as a (rows, k) int32 numpy array (row-major)."""
    info = tid_set_info(set_)
    rows = tid_set_rows(set_)
    if buf is None:
        buf = np.empty((rows, info["cols"]), np.int32)
    elif (not isinstance(buf, np.ndarray) or buf.dtype != np.int32 or buf.ndim != 2
          or buf.shape[1] != info["cols"] or not buf.flags["C_CONTIGUOUS"]):
        raise ValueError(f"buf must be a C-contiguous int32 array of shape (rows, {info['cols']})")
    got = C.c_int64()
    _check(lib().tid_set_to_host(set_, _ptr(buf) if buf.size else None, buf.shape[0], C.byref(got)),
           "tid_set_to_host")
    return buf[:got.value]


def tid_set_free(set_):
    _check(lib().tid_set_free(set_), "tid_set_free")


def _preds(preds):
    preds = list(preds or [])
    arr = (tid_pred * max(1, len(preds)))()
    for i, q in enumerate(preds):
        if isinstance(q, dict):
            var, op, a, b = q["var"], q["cmp"], q["a"], q.get("b", 0)
        else:
            var, op, a, b = (tuple(q) + (0,))[:4]
        arr[i].var, arr[i].op = int(var), CMP[op] if isinstance(op, str) else int(op)
        arr[i].a, arr[i].b = int(a), int(b)
    return arr, len(preds)


def tid_match_noalloc(device, stream, s, p, o, pattern, out, count, n=None, cap=None):
    """tid_match into caller buffers, allocating nothing (torch CUDA tensors or raw
    device addresses; stream as int or None)."""
    n = int(s.shape[0]) if n is None else int(n)
    cap = int(out.shape[0]) if cap is None else int(cap)
    for c in (s, p, o, out):
        _int_dtype(c, "columns and out", 32)
    _int_dtype(count, "count", 64)
    _within(n, "n", s, p, o)
    _within(cap, "cap", out)
    _within(1, "count", count)
    _check(lib().tid_match_noalloc(int(device), stream if stream else None, _ptr(s), _ptr(p), _ptr(o), n,
                                   as_pattern(pattern), _ptr(out), cap, _ptr(count)), "tid_match_noalloc")


def tid_match_multi(ctx, st, patterns):
    pats = [as_pattern(p) for p in patterns]
    arr = (tid_pattern * len(pats))(*pats)
    outs = (_vp * len(pats))()
    _check(lib().tid_match_multi(ctx, st, arr, len(pats), outs), "tid_match_multi")
    return [_vp(outs[i]) for i in range(len(pats))]


PATTERN_DTYPE = np.dtype([("s", "<i4"), ("p", "<i4"), ("o", "<i4"), ("var", "i1", (3,)), ("reserved", "i1")])


def pattern_array(patterns):
    """Patterns as a packed tid_pattern array (numpy): from an (q, 3) integer array
    of keys (anonymous variables), or from a list of anything as_pattern takes."""
    if isinstance(patterns, np.ndarray) and patterns.dtype == PATTERN_DTYPE:
        return patterns
    if isinstance(patterns, np.ndarray) and patterns.ndim == 2 and patterns.shape[1] == 3:
        arr = np.zeros(patterns.shape[0], PATTERN_DTYPE)
        arr["s"], arr["p"], arr["o"] = patterns[:, 0], patterns[:, 1], patterns[:, 2]
        arr["var"] = -1
        return arr
    arr = np.zeros(len(patterns), PATTERN_DTYPE)
    for i, x in enumerate(patterns):
        t = as_pattern(x)
        arr[i] = (t.s, t.p, t.o, tuple(t.var), 0)
    return arr


def tid_match_batch(ctx, st, patterns):
    """Index lists of many patterns (see tid.h); `patterns` as pattern_array takes."""
    arr = pattern_array(patterns)
    q = int(arr.shape[0])
    outs = (_vp * max(1, q))()
    ptr = arr.ctypes.data_as(C.POINTER(tid_pattern)) if q else None
    _check(lib().tid_match_batch(ctx, st, ptr, q, outs), "tid_match_batch")
    return [_vp(outs[i]) for i in range(q)]


BATCH_SHAPES = {0: "direct", 1: "direct_skip", 2: "queue4", 3: "queue8"}


def tid_batch_tuning(ctx):
    """The autotuner's choice for the context's last batched search (see tid.h)."""
    sh, keys, subs = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().tid_batch_tuning(ctx, C.byref(sh), C.byref(keys), C.byref(subs)), "tid_batch_tuning")
    return {"shape": BATCH_SHAPES.get(sh.value, None), "keys_per_sub_batch": keys.value, "sub_batches": subs.value}


def tid_batch_table_check(patterns, seed):
    """Host-only check of tid_match_batch's key tables (see tid.h): returns
    (status, table builds tried, sub-batches)."""
    arr = pattern_array(patterns)
    q = int(arr.shape[0])
    ptr = arr.ctypes.data_as(C.POINTER(tid_pattern)) if q else None
    tries, subs = C.c_int(0), C.c_int(0)
    rc = int(lib().tid_batch_table_check(ptr, q, int(seed) & 0xFFFFFFFF, C.byref(tries), C.byref(subs)))
    return rc, int(tries.value), int(subs.value)


def tid_bind(ctx, st, pattern, idx, preds=()):
    arr, n = _preds(preds)
    out = _vp()
    _check(lib().tid_bind(ctx, st, as_pattern(pattern), idx, arr, n, C.byref(out)), "tid_bind")
    return out


def tid_filter(ctx, set_, preds):
    arr, n = _preds(preds)
    out = _vp()
    _check(lib().tid_filter(ctx, set_, arr, n, C.byref(out)), "tid_filter")
    return out


def tid_join(ctx, L, R, algo="auto"):
    out = _vp()
    _check(lib().tid_join(ctx, L, R, JOIN[algo] if isinstance(algo, str) else int(algo), C.byref(out)),
           "tid_join")
    return out


def tid_union(ctx, sets):
    arr = (_vp * len(sets))(*[s.value if isinstance(s, _vp) else s for s in sets])
    out = _vp()
    _check(lib().tid_union(ctx, arr, len(sets), C.byref(out)), "tid_union")
    return out


def tid_project(ctx, set_, vars_):
    arr = (C.c_int8 * max(1, len(vars_)))(*[int(v) for v in vars_])
    out = _vp()
    _check(lib().tid_project(ctx, set_, arr, len(vars_), C.byref(out)), "tid_project")
    return out


def tid_set_from_host(ctx, rows, vars_):
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    if rows.ndim != 2 or rows.shape[1] != len(vars_):
        raise ValueError("rows must be (n, len(vars))")
    arr = (C.c_int8 * len(vars_))(*[int(v) for v in vars_])
    out = _vp()
    _check(lib().tid_set_from_host(ctx, rows.ctypes.data if rows.size else None, rows.shape[0],
                                   rows.shape[1], arr, C.byref(out)), "tid_set_from_host")
    return out


def plan_nodes(plan):
    """A plan given as a list of dicts (op, pattern / input(s) / var, cmp, a, b /
    algo / vars) as a tid_plan_node array."""
    nodes = (tid_plan_node * len(plan))()
    for i, nd in enumerate(plan):
        x = nodes[i]
        x.op = OP[nd["op"]]
        ins = nd.get("inputs", [nd["input"]] if "input" in nd else [])
        x.n_in = len(ins)
        for j, v in enumerate(ins):
            x.in_[j] = int(v)
        if nd["op"] == "match":
            x.pattern = as_pattern(nd["pattern"])
        if nd["op"] == "filter":
            p, _ = _preds([nd])
            x.pred = p[0]
        if nd["op"] == "join":
            a = nd.get("algo", "auto")
            x.algo = JOIN[a] if isinstance(a, str) else int(a)
        if nd["op"] == "project":
            x.n_vars = len(nd["vars"])
            for j, v in enumerate(nd["vars"]):
                x.vars[j] = int(v)
    return nodes


def tid_plan_check(plan) -> int:
    """Status code of the checks tid_exec makes before running a plan (no GPU)."""
    nodes = plan if isinstance(plan, C.Array) else plan_nodes(plan)
    return int(lib().tid_plan_check(nodes, len(nodes)))


def tid_exec(ctx, st, plan):
    nodes = plan if isinstance(plan, C.Array) else plan_nodes(plan)
    out = _vp()
    _check(lib().tid_exec(ctx, st, nodes, len(nodes), C.byref(out)), "tid_exec")
    return out


# ---------------------------------------------------------------------------
# small conveniences (no computation)
# ---------------------------------------------------------------------------

class Context:
    """Owns a tid_ctx; frees the stores and sets made through it on close()."""

    def __init__(self, device=0, stream=None):
        self.h = tid_ctx_create(device, stream)
        self._owned = []

    def load(self, s, p, o, **kw):
        st = tid_load(self.h, s, p, o, **kw)
        self._owned.append(("store", st))
        return st

    def track(self, set_):
        self._owned.append(("set", set_))
        return set_

    def sync(self):
        tid_ctx_sync(self.h)

    def close(self):
        for kind, h in reversed(self._owned):
            (tid_store_free if kind == "store" else tid_set_free)(h)
        self._owned = []
        if self.h:
            tid_ctx_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def tid_ctx_test_bounded_wait(ctx, polls):
    """Status code of a bounded in-kernel wait that nothing ends (see tid.h):
    TID_ERR_TIMEOUT when the wait gave up as it should."""
    return int(lib().tid_ctx_test_bounded_wait(ctx, int(polls)))


def tid_ctx_inject_alloc_failure(ctx, after):
    """After `after` more device allocations on ctx, fail the rest with TID_ERR_OOM (< 0: off)."""
    _check(lib().tid_ctx_inject_alloc_failure(ctx, int(after)), "tid_ctx_inject_alloc_failure")


def tid_entail(ctx, st, rule, vocab):
    """Conclusions of RDFS rule `rule` (2, 3, 5, 7, 9, 11) as a 3-column set (s, p, o),
    and the step counts; vocab: dict with type, domain, range, subprop, subclass IDs."""
    v = tid_rdfs_vocab(int(vocab["type"]), int(vocab["domain"]), int(vocab["range"]),
                       int(vocab["subprop"]), int(vocab["subclass"]))
    out, stats = _vp(), tid_entail_stats()
    _check(lib().tid_entail(ctx, st, int(rule), C.byref(v), C.byref(out), C.byref(stats)), "tid_entail")
    return out, {f: getattr(stats, f) for f, _ in tid_entail_stats._fields_}


class Server:
    """A tid_server over device columns s, p, o (kept referenced while it lives).
    Requests: submit_index(pattern) -> ascending index list; submit_plan(plan)
    -> canonical tuple set (rows x vars).  See tid.h for the scheduling rules."""

    def __init__(self, s, p, o, device=0, workers=2, max_wave=4096, batch_scans=True, budget_bytes=60 << 30):
        self._cols = (s, p, o)
        cfg = tid_server_config(int(workers), int(max_wave), 1 if batch_scans else 0, 0, int(budget_bytes))
        h = _vp()
        n = int(s.shape[0])
        for c in (s, p, o):
            _int_dtype(c, "store columns", 32)
            if not (hasattr(c, "is_cuda") and c.is_cuda):
                raise TypeError("the server borrows device columns (torch CUDA tensors)")
        _within(n, "n", p, o)
        _check(lib().tid_server_create(int(device), _ptr(s), _ptr(p), _ptr(o), n, C.byref(cfg), C.byref(h)),
               "tid_server_create")
        self.h = h

    @staticmethod
    def now_ns() -> int:
        return int(lib().tid_server_now_ns())

    def _submit(self, kind, nodes, arrival_ns):
        rid = C.c_int64()
        _check(lib().tid_server_submit(self.h, kind, nodes, len(nodes), int(arrival_ns), C.byref(rid)),
               "tid_server_submit")
        return rid.value

    @staticmethod
    def request(kind, x):
        """(kind code, node array) of an index request (x: a pattern) or a plan request
        (x: a plan), prepared ahead of submission."""
        if kind == "index":
            nodes = (tid_plan_node * 1)()
            nodes[0].op = OP["match"]
            nodes[0].pattern = as_pattern(x)
            return TID_REQ_INDEX, nodes
        return TID_REQ_PLAN, plan_nodes(x)

    def submit(self, prepared, arrival_ns=0):
        return self._submit(prepared[0], prepared[1], arrival_ns)

    def submit_index(self, pattern, arrival_ns=0):
        return self.submit(self.request("index", pattern), arrival_ns)

    def submit_plan(self, plan, arrival_ns=0):
        return self.submit(self.request("plan", plan), arrival_ns)

    def wait(self, rid, timeout_ms=-1) -> bool:
        rc = lib().tid_server_wait(self.h, int(rid), int(timeout_ms))
        if rc == TID_ERR_TIMEOUT:
            return False
        _check(rc, "tid_server_wait")
        return True

    def result(self, rid, release=True):
        """(status, vars, rows array (rows x cols int32, a copy), latency in ns)."""
        st, k, rows, lat = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
        vars_ = (C.c_int8 * TID_MAX_COLS)()
        data = C.POINTER(C.c_int32)()
        _check(lib().tid_server_result(self.h, int(rid), C.byref(st), C.byref(k), vars_, C.byref(rows),
                                       C.byref(data), C.byref(lat)), "tid_server_result")
        n = rows.value * k.value
        arr = np.ctypeslib.as_array(data, shape=(n,)).copy() if n else np.zeros(0, np.int32)
        out = (st.value, tuple(vars_[:k.value]), arr.reshape(rows.value, max(1, k.value)), lat.value)
        if release:
            self.release(rid)
        return out

    def release(self, rid):
        _check(lib().tid_server_release(self.h, int(rid)), "tid_server_release")

    def stats(self) -> dict:
        st = tid_server_stats()
        _check(lib().tid_server_get_stats(self.h, C.byref(st)), "tid_server_get_stats")
        return {f: getattr(st, f) for f, _ in tid_server_stats._fields_}

    def close(self):
        if self.h:
            lib().tid_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
