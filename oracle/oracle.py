"""TripleID-Q CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct CPU statement of what the query hot path
computes, used to check the CUDA library result by result.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA path: the loops live in ``oracle.c``
(compiled here with gcc, loaded with ctypes) and the set algebra around them in
numpy below.  Tuple sets are row-major (rows x k) int32 arrays with one
variable id per column.

Paper passages followed (TripleID-Q, IEEE TPDS 2018):
* ``match``        -- Section 3, Algorithm 1 and its brute-force GPUSearch test;
                      key value 0 is the free variable "?".
* ``match_multi``  -- Section 4.1, keysArray / positionArray[i].query.
* ``bind``         -- Section 4.2, result vectors R_qi (terms at the variable slots).
* ``join``         -- Section 4.2 steps 1-3 and the relationship table (shared term
                      at any of S/P/O on either side); inner join.
* ``left_join``    -- the left (outer) join Section 4.2 names among its library's joins:
                      SPARQL OPTIONAL, unmatched left rows padded with 0.
* ``right_join``, ``full_join`` -- the right and full outer joins of the same list:
                      unmatched right rows (and, for full, left rows) padded with 0.
* ``union``        -- Section 4.1; results keep only distinct values (Section 4.3).
* ``filter``       -- Section 4.3 (filter during extraction), on integer IDs with the
                      order-preserving literal encoding the same section proposes.
* ``project``      -- Section 4.3, SELECT variables and DISTINCT.
* ``execute``      -- Section 4.3 / Fig. "Integration of several operations": per
                      subquery search+extract (filter fused), joins left to right,
                      distinct results.
* ``entail``       -- Section 5, Table "RDFS Entailment rules" (R2, R3, R5, R7, R9,
                      R11) and the Rule-11 walk-through: search the schema premise,
                      keep its distinct join terms, search the store for the triples
                      whose term at the join position is one of them (the keysArray
                      of the second GPUSearch), join the two result vectors on the
                      shared term, keep the distinct conclusions.

Readings where the paper is silent: 0 (unbound, e.g. union padding) never joins
and never passes a filter; every result is a set in canonical order (rows
sorted lexicographically by column order, duplicates removed).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

OPS = {"eq": 0, "ne": 1, "lt": 2, "le": 3, "gt": 4, "ge": 5, "range": 6}
NESTED_LOOP_CAP = 100_000_000  # |L|*|R| above this switches to the sort-merge join
JOIN_PATHS = {"nested": 0, "sortmerge": 0}  # joins run per path, for the parity log

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (plain gcc, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = f"{_SO}.{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Run the oracle on another build of oracle.c (the pin tests use this to
    show that planted mistakes are caught)."""
    global _lib
    saved = _lib
    _lib = _load(path)
    try:
        yield
    finally:
        _lib = saved


def _load(path):
    L = C.CDLL(path)
    i32p, i64p = C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    L.or_match.restype = C.c_int64
    L.or_match.argtypes = [i32p, i32p, i32p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, i32p]
    L.or_match_multi.restype = None
    L.or_match_multi.argtypes = [i32p, i32p, i32p, C.c_int64, i32p, C.c_int, i64p,
                                 C.POINTER(i32p)]
    L.or_bind.restype = C.c_int64
    L.or_bind.argtypes = [i32p, i32p, i32p, i32p, C.c_int64, C.c_char_p, C.c_int,
                          C.c_char_p, i32p]
    L.or_canonical.restype = C.c_int64
    L.or_canonical.argtypes = [i32p, C.c_int64, C.c_int]
    ip = C.POINTER(C.c_int)
    for f in (L.or_join_nested, L.or_join_sortmerge):
        f.restype = C.c_int64
        f.argtypes = [i32p, C.c_int64, C.c_int, i32p, C.c_int64, C.c_int,
                      C.c_int, ip, ip, C.c_int, ip, i32p]
    L.or_filter.restype = C.c_int64
    L.or_filter.argtypes = [i32p, C.c_int64, C.c_int, C.c_int, C.c_int,
                            C.c_int32, C.c_int32, i32p]
    return L


def _p32(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _ints(xs):
    arr = (C.c_int * max(1, len(xs)))(*xs)
    return arr


def _col(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------------------
# tuple sets
# ---------------------------------------------------------------------------

@dataclass
class TupleSet:
    vars: tuple          # variable id per column
    rows: np.ndarray     # (n, k) int32, row-major

    @property
    def n(self):
        return int(self.rows.shape[0])

    @property
    def k(self):
        return len(self.vars)


def canonical(rows: np.ndarray) -> np.ndarray:
    """Rows sorted lexicographically in column order, duplicates removed."""
    rows = np.array(rows, dtype=np.int32, order="C", copy=True)
    if rows.ndim != 2:
        raise ValueError("rows must be 2-D")
    n, k = rows.shape
    if n == 0 or k == 0:
        return rows
    m = lib().or_canonical(_p32(rows), n, k)
    if m < 0:
        raise MemoryError("oracle canonical: out of memory")
    return rows[:m].copy()


def _set(vars_, rows):
    return TupleSet(tuple(int(v) for v in vars_), canonical(rows))


# ---------------------------------------------------------------------------
# search
# ---------------------------------------------------------------------------

def match(s, p, o, key) -> np.ndarray:
    """Ascending positions i with (S[i], P[i], O[i]) answering key (0 = "?")."""
    s, p, o = _col(s), _col(p), _col(o)
    ks, kp, ko = (int(x) for x in key)
    if min(ks, kp, ko) < 0:
        raise ValueError("negative ID in a key")
    L = lib()
    h = L.or_match(_p32(s), _p32(p), _p32(o), s.shape[0], ks, kp, ko, None)
    out = np.empty(h, np.int32)
    L.or_match(_p32(s), _p32(p), _p32(o), s.shape[0], ks, kp, ko, _p32(out))
    return out


def match_multi(s, p, o, keys) -> list:
    """One pass over the store for m keys; one ascending position list per key."""
    s, p, o = _col(s), _col(p), _col(o)
    keys = np.ascontiguousarray(np.asarray(keys, dtype=np.int32).reshape(-1, 3))
    m = keys.shape[0]
    if m == 0:
        return []
    if keys.min() < 0:
        raise ValueError("negative ID in a key")
    L = lib()
    counts = np.zeros(m, np.int64)
    L.or_match_multi(_p32(s), _p32(p), _p32(o), s.shape[0], _p32(keys), m,
                     counts.ctypes.data_as(C.POINTER(C.c_int64)), None)
    outs = [np.empty(int(c), np.int32) for c in counts]
    ptrs = (C.POINTER(C.c_int32) * m)(*[_p32(x) for x in outs])
    L.or_match_multi(_p32(s), _p32(p), _p32(o), s.shape[0], _p32(keys), m,
                     counts.ctypes.data_as(C.POINTER(C.c_int64)), ptrs)
    return outs


def pattern_vars(key, var) -> tuple:
    """Output variables of a pattern: distinct ids at its "?" slots, in s,p,o order."""
    out = []
    for j in range(3):
        v = int(var[j])
        if v < 0:
            continue
        if int(key[j]) != 0:
            raise ValueError("a bound slot cannot carry a variable")
        if v not in out:
            out.append(v)
    if not out:
        raise ValueError("pattern has no variable")
    if len(out) > 8:
        raise ValueError("too many variables")
    return tuple(out)


def bind(s, p, o, key, var, idx) -> TupleSet:
    """Result vector of one subquery: values at the variable slots of each hit."""
    s, p, o = _col(s), _col(p), _col(o)
    idx = _col(idx)
    vars_ = pattern_vars(key, var)
    k = len(vars_)
    out = np.empty((idx.shape[0], k), np.int32)
    vb = bytes((int(v) & 0xFF) for v in var)
    ob = bytes((int(v) & 0xFF) for v in vars_)
    r = lib().or_bind(_p32(s), _p32(p), _p32(o), _p32(idx), idx.shape[0], vb, k, ob, _p32(out))
    return _set(vars_, out[:r])


# ---------------------------------------------------------------------------
# operators on tuple sets
# ---------------------------------------------------------------------------

def join_schema(Lv, Rv):
    shared = [v for v in Lv if v in Rv]
    lkey = [Lv.index(v) for v in shared]
    rkey = [Rv.index(v) for v in shared]
    rrest = [j for j, v in enumerate(Rv) if v not in Lv]
    out_vars = tuple(Lv) + tuple(Rv[j] for j in rrest)
    return shared, lkey, rkey, rrest, out_vars


def join(Ls: TupleSet, Rs: TupleSet, method: str = "auto") -> TupleSet:
    """Inner join on all shared variables; output = L's columns then R's others."""
    shared, lkey, rkey, rrest, out_vars = join_schema(Ls.vars, Rs.vars)
    if len(out_vars) > 8:
        raise ValueError("join output wider than 8 columns")
    if method == "auto":
        method = "nested" if Ls.n * Rs.n <= NESTED_LOOP_CAP else "sortmerge"
    f = {"nested": lib().or_join_nested, "sortmerge": lib().or_join_sortmerge}[method]
    JOIN_PATHS[method] += 1
    Lr = np.ascontiguousarray(Ls.rows, np.int32)
    Rr = np.ascontiguousarray(Rs.rows, np.int32)
    args = (_p32(Lr), Ls.n, Ls.k, _p32(Rr), Rs.n, Rs.k, len(shared),
            _ints(lkey), _ints(rkey), len(rrest), _ints(rrest))
    m = f(*args, None)
    if m < 0:
        raise MemoryError("oracle join: out of memory")
    out = np.empty((m, len(out_vars)), np.int32)
    f(*args, _p32(out))
    return _set(out_vars, out)


def left_join(Ls: TupleSet, Rs: TupleSet, method: str = "auto") -> TupleSet:
    """Left outer join (OPTIONAL; Section 4.2 names the left and outer joins of the
    library the paper used): the inner join's rows, plus every row of L that joins
    no row of R, with R's other columns 0 (unbound)."""
    inner = join(Ls, Rs, method)
    shared, lkey, rkey, rrest, out_vars = join_schema(Ls.vars, Rs.vars)
    rkeys = {tuple(r[j] for j in rkey) for r in Rs.rows.tolist() if all(r[j] != 0 for j in rkey)}
    pad = [l + [0] * len(rrest) for l in Ls.rows.tolist()
           if not (all(l[i] != 0 for i in lkey) and tuple(l[i] for i in lkey) in rkeys)]
    rows = np.concatenate([inner.rows, np.array(pad, np.int32).reshape(-1, len(out_vars))], axis=0)
    return _set(out_vars, rows)


def _unmatched_right(Ls: TupleSet, Rs: TupleSet):
    """Rows of R that join no row of L, in the join's columns (L's, then R's
    others), L's other columns 0 (unbound)."""
    shared, lkey, rkey, rrest, out_vars = join_schema(Ls.vars, Rs.vars)
    lkeys = {tuple(l[i] for i in lkey) for l in Ls.rows.tolist() if all(l[i] != 0 for i in lkey)}
    pad = []
    for r in Rs.rows.tolist():
        key = tuple(r[j] for j in rkey)
        if all(x != 0 for x in key) and key in lkeys:
            continue
        pad.append([r[Rs.vars.index(v)] if v in Rs.vars else 0 for v in out_vars])
    return np.array(pad, np.int32).reshape(-1, len(out_vars))


def right_join(Ls: TupleSet, Rs: TupleSet, method: str = "auto") -> TupleSet:
    """Right outer join (Section 4.2 names the outer joins of the library the paper
    used): the inner join's rows, plus every row of R that joins no row of L, with
    L's other columns 0 (unbound); columns as the inner join's."""
    inner = join(Ls, Rs, method)
    return _set(inner.vars, np.concatenate([inner.rows, _unmatched_right(Ls, Rs)], axis=0))


def full_join(Ls: TupleSet, Rs: TupleSet, method: str = "auto") -> TupleSet:
    """Full outer join: the inner join's rows, every row of L that joins no row of
    R (R's other columns 0) and every row of R that joins no row of L (L's other
    columns 0)."""
    left = left_join(Ls, Rs, method)
    return _set(left.vars, np.concatenate([left.rows, _unmatched_right(Ls, Rs)], axis=0))


def union_schema(sets):
    out = []
    for t in sets:
        for v in t.vars:
            if v not in out:
                out.append(v)
    return tuple(out)


def union(sets) -> TupleSet:
    """Set union; branches with other variables are padded with 0 (unbound)."""
    sets = list(sets)
    if not sets:
        raise ValueError("union of nothing")
    uv = union_schema(sets)
    if len(uv) > 8:
        raise ValueError("union schema wider than 8 columns")
    parts = []
    for t in sets:
        a = np.zeros((t.n, len(uv)), np.int32)
        for j, v in enumerate(t.vars):
            a[:, uv.index(v)] = t.rows[:, j]
        parts.append(a)
    return _set(uv, np.concatenate(parts, axis=0))


def filter(t: TupleSet, var: int, op: str, a: int, b: int = 0) -> TupleSet:
    """Rows whose value of var passes the comparison (0 = unbound never passes)."""
    if var not in t.vars:
        raise ValueError("filter variable not in the set")
    rows = np.ascontiguousarray(t.rows, np.int32)
    out = np.empty_like(rows)
    m = lib().or_filter(_p32(rows), t.n, t.k, t.vars.index(var), OPS[op], int(a), int(b),
                        _p32(out))
    return TupleSet(t.vars, out[:m].copy())


def project(t: TupleSet, vars_) -> TupleSet:
    """SELECT the given variables (in that order) with DISTINCT."""
    cols = [t.vars.index(v) for v in vars_]
    return _set(vars_, t.rows[:, cols])


# ---------------------------------------------------------------------------
# plans
# ---------------------------------------------------------------------------

def execute(s, p, o, plan) -> TupleSet:
    """Evaluate a plan (list of node dicts; the last node is the root)."""
    memo = {}

    def ev(i):
        if i in memo:
            return memo[i]
        nd = plan[i]
        op = nd["op"]
        if op == "match":
            pat = nd["pattern"]
            idx = match(s, p, o, pat.key())
            r = bind(s, p, o, pat.key(), pat.var, idx)
        elif op == "filter":
            r = filter(ev(nd["input"]), nd["var"], nd["cmp"], nd["a"], nd.get("b", 0))
        elif op == "join":
            a, b = nd["inputs"]
            kind = {"left": left_join, "right": right_join, "full": full_join}.get(nd.get("algo"), join)
            r = kind(ev(a), ev(b))
        elif op == "union":
            r = union([ev(j) for j in nd["inputs"]])
        elif op == "project":
            r = project(ev(nd["input"]), tuple(nd["vars"]))
        else:
            raise ValueError(f"unknown plan op {op}")
        memo[i] = r
        return r

    return ev(len(plan) - 1)


# ---------------------------------------------------------------------------
# RDFS entailment (Section 5)
# ---------------------------------------------------------------------------

# The six two-premise rules of the table, written as premise patterns over
# variable names and fixed vocabulary terms, the shared variable, and the
# conclusion.  Premise 1 is the schema triple (searched first), premise 2 the
# data triple (searched with the distinct values of the shared variable).
ENTAIL_RULES = {
    2: {"schema": ("p", "domain", "D"), "data": ("s", "p", "o"), "on": "p", "then": ("s", "type", "D")},
    3: {"schema": ("p", "range", "R"), "data": ("s", "p", "o"), "on": "p", "then": ("o", "type", "R")},
    5: {"schema": ("p", "subprop", "q"), "data": ("q", "subprop", "r"), "on": "q", "then": ("p", "subprop", "r")},
    7: {"schema": ("p", "subprop", "q"), "data": ("s", "p", "o"), "on": "p", "then": ("s", "q", "o")},
    9: {"schema": ("x", "subclass", "y"), "data": ("s", "type", "x"), "on": "x", "then": ("s", "type", "y")},
    11: {"schema": ("x", "subclass", "y"), "data": ("y", "subclass", "z"), "on": "y", "then": ("x", "subclass", "z")},
}
VOCAB_TERMS = ("type", "domain", "range", "subprop", "subclass")


def entail(s, p, o, rule: int, vocab: dict):
    """Conclusions of one rule over the store, as a set of (s, p, o) rows (vars
    0, 1, 2), plus the step counts of the paper's table: res1 (matches of the
    schema premise), dist1 (its distinct join terms), res2 (store triples found
    by the second search), dist2 (their distinct join terms), all (conclusions)."""
    s, p, o = _col(s), _col(p), _col(o)
    r = ENTAIL_RULES[rule]
    names = {}

    def pattern(tpl):
        key, var = [], []
        for j, t in enumerate(tpl):
            if t in VOCAB_TERMS:
                key.append(int(vocab[t]))
                var.append(-1)
            else:
                names.setdefault(t, len(names))
                key.append(0)
                var.append(names[t])
        return key, var

    k1, v1 = pattern(r["schema"])
    k2, v2 = pattern(r["data"])
    on = names[r["on"]]
    # step 1: the schema premise; its distinct join terms become the keys of step 2
    idx1 = match(s, p, o, k1)
    t1 = bind(s, p, o, k1, v1, idx1)
    keys = np.unique(t1.rows[:, t1.vars.index(on)]) if t1.n else np.zeros(0, np.int32)
    # step 2: the triples of premise 2 whose term at the join slot is one of the keys
    slot = r["data"].index(r["on"])
    cand = match(s, p, o, k2)
    col = (s, p, o)[slot]
    idx2 = cand[np.isin(col[cand], keys)] if cand.shape[0] else cand
    t2 = bind(s, p, o, k2, v2, idx2)
    dist2 = int(np.unique(t2.rows[:, t2.vars.index(on)]).shape[0]) if t2.n else 0
    # combine: join on the shared term, the conclusion's terms, distinct
    j = join(t1, t2)
    cols = []
    for t in r["then"]:
        if t in VOCAB_TERMS:
            cols.append(np.full(j.n, int(vocab[t]), np.int32))
        else:
            cols.append(j.rows[:, j.vars.index(names[t])])
    rows = np.stack(cols, axis=1) if j.n else np.zeros((0, 3), np.int32)
    out = _set((0, 1, 2), rows)
    stats = {"res1": int(idx1.shape[0]), "dist1": int(keys.shape[0]), "res2": int(idx2.shape[0]),
             "dist2": dist2, "all": out.n}
    return out, stats
