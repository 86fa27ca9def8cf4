"""Tuple-set operators through the C ABI against the CPU oracle, bit-exact:
multi-pattern scan (K2), bind with fused filters (K3), filter, canonical sort
(K4), sort-merge and hash joins (K5/K6) in every relationship type of the
paper's table, union with schema padding (K7), project, and whole plans."""
import itertools
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import pins
from paper_1807_01409_gb300 import binding as tb
from paper_1807_01409_gb300 import synth

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    from paper_1807_01409_gb300 import build
    build.build()
    c = tb.tid_ctx_create(0, None)
    yield c
    tb.tid_ctx_destroy(c)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def _host(h, free=True):
    try:
        info = tb.tid_set_info(h)
        return info["vars"], tb.tid_set_to_host(h).copy()
    finally:
        if free:
            tb.tid_set_free(h)


def _store(ctx, S, P, O):
    return tb.tid_load(ctx, _dev(S), _dev(P), _dev(O), copy=1)


def _same(got, want):
    gv, gr = got
    assert tuple(gv) == tuple(want.vars), (gv, want.vars)
    assert gr.shape == want.rows.shape, (gr.shape, want.rows.shape)
    assert np.array_equal(gr, want.rows)


# ---------------------------------------------------------------- K2 multi-match

@pytest.mark.parametrize("n", [0, 7, 4096, 5000, 100_003])
def test_match_multi_equals_single(ctx, orc, n):
    rng = np.random.default_rng(n + 1)
    S = rng.integers(1, 6, n).astype(np.int32)
    P = rng.integers(1, 4, n).astype(np.int32)
    O = rng.integers(1, 7, n).astype(np.int32)
    st = _store(ctx, S, P, O)
    keys = [(1, 0, 0), (0, 2, 0), (0, 0, 3), (1, 2, 0), (0, 2, 3), (4, 0, 5), (2, 3, 1), (0, 0, 0),
            (0, 2, 0), (5, 1, 6), (3, 0, 0), (0, 1, 0), (0, 3, 2), (9, 0, 0), (1, 1, 1), (2, 0, 2)]
    for m in (1, 2, 5, 16):
        hs = tb.tid_match_multi(ctx, st, keys[:m])
        want = orc.match_multi(S, P, O, keys[:m])
        for h, w in zip(hs, want):
            assert np.array_equal(tb.tid_set_to_host(h)[:, 0], w)
            tb.tid_set_free(h)
    tb.tid_store_free(st)


def test_match_multi_worked_example(ctx):
    g = json.load(open(os.path.join(GOLDEN, "rule11_worked_example.json")))
    a = np.array(g["store"], np.int32)
    st = _store(ctx, a[:, 0], a[:, 1], a[:, 2])
    flags = np.zeros(len(a), int)
    for h in tb.tid_match_multi(ctx, st, [tuple(k) for k in g["step2"]["keys"]]):
        flags[tb.tid_set_to_host(h)[:, 0]] = 1
        tb.tid_set_free(h)
    assert flags.tolist() == g["step2"]["flags"]
    tb.tid_store_free(st)


# ---------------------------------------------------------------- K3 bind / filter

def test_bind_with_fused_filters_tiny_store(ctx, orc):
    st_np = synth.tiny_store()
    st = _store(ctx, st_np.s, st_np.p, st_np.o)
    X, Y, Z = 0, 1, 2
    cases = [((0, 2, 0), (X, -1, Y), []),
             ((0, 1, 0), (X, -1, Y), [(Y, "range", 10, 500)]),
             ((0, 0, 0), (X, Y, Z), [(Y, "le", 3), (Z, "gt", 1000)]),
             ((0, 3, 0), (X, -1, X), []),                    # repeated variable
             ((0, 2, 0), (X, -1, -1), []),                   # anonymous slot: duplicates removed
             ((77, 0, 0), (-1, X, Y), [(X, "ne", 1)])]
    for key, var, preds in cases:
        idx = tb.tid_match(ctx, st, key)
        h = tb.tid_bind(ctx, st, (*key, var), idx, preds)
        tb.tid_set_free(idx)
        want = orc.bind(st_np.s, st_np.p, st_np.o, key, var, orc.match(st_np.s, st_np.p, st_np.o, key))
        for v, op, *ab in preds:
            want = orc.filter(want, v, op, *ab)
        _same(_host(h), want)
    tb.tid_store_free(st)


@pytest.mark.parametrize("order", ["spo", "shuffled", "one_swap"])
def test_bind_store_order(ctx, orc, order):
    """In a store sorted by (s, p, o), bind keeps index order (no sort) when no
    anonymous slot precedes a variable, and drops adjacent repeats when one
    follows them.  The same triples shuffled, or with one adjacent pair
    swapped (the load's order check must see a single inversion), take the
    sorting path.  Every pattern shape, with and without a fused filter, gives
    the oracle's rows."""
    rng = np.random.default_rng(11)
    n = 200_000
    keys = np.unique(np.stack([rng.integers(1, 3000, n), rng.integers(1, 9, n), rng.integers(1, 3000, n)], 1),
                     axis=0)
    if order == "shuffled":
        keys = keys[rng.permutation(len(keys))]
    elif order == "one_swap":
        i = len(keys) // 2
        keys[[i, i + 1]] = keys[[i + 1, i]]
    S, P, O = (keys[:, j].astype(np.int32).copy() for j in range(3))
    st = _store(ctx, S, P, O)
    X, Y, Z = 0, 1, 2
    cases = [((0, 3, 0), (X, -1, Y), []),
             ((0, 3, 0), (X, -1, Y), [(Y, "lt", 1500)]),
             ((0, 0, 0), (X, Y, Z), []),
             ((0, 0, 0), (X, -1, Y), []),                    # anonymous between the variables
             ((0, 0, 0), (X, Y, -1), []),                    # anonymous last: adjacent repeats
             ((0, 0, 0), (X, Y, -1), [(X, "ge", 100)]),
             ((0, 0, 0), (-1, X, Y), []),                    # anonymous first
             ((0, 5, 0), (X, -1, X), []),                    # repeated variable
             ((7, 0, 0), (-1, X, Y), []),
             ((0, 0, 11), (X, Y, -1), []),
             ((0, 4, 0), (Y, -1, X), [])]                    # column order follows the slots, not the ids
    for key, var, preds in cases:
        idx = tb.tid_match(ctx, st, key)
        h = tb.tid_bind(ctx, st, (*key, var), idx, preds)
        tb.tid_set_free(idx)
        want = orc.bind(S, P, O, key, var, orc.match(S, P, O, key))
        for v, op, *ab in preds:
            want = orc.filter(want, v, op, *ab)
        _same(_host(h), want)
    tb.tid_store_free(st)


@pytest.mark.parametrize("n", [0, 1, 2047, 2048, 2049, 30_001])
def test_filter_all_ops(ctx, orc, n):
    rng = np.random.default_rng(n)
    rows = orc.canonical(rng.integers(-5, 60, (n, 3)))
    want_set = orc.TupleSet((3, 1, 4), rows)
    h = tb.tid_set_from_host(ctx, rows, (3, 1, 4))
    for op, a, b in [("eq", 7, 0), ("ne", 7, 0), ("lt", 20, 0), ("le", 20, 0), ("gt", 20, 0), ("ge", 20, 0),
                     ("range", 5, 40), ("range", 40, 5), ("lt", -1, 0)]:
        for var in (3, 1, 4):
            f = tb.tid_filter(ctx, h, [(var, op, a, b)])
            _same(_host(f), orc.filter(want_set, var, op, a, b))
    tb.tid_set_free(h)


# ---------------------------------------------------------------- K4 canonical sort

@pytest.mark.parametrize("n,k,hi", [(0, 1, 5), (1, 2, 5), (4095, 1, 1 << 30), (4097, 3, 9), (70_000, 2, 300),
                                    (200_001, 4, 1 << 31), (50_000, 8, 4), (123_457, 1, 2)])
def test_canonical_sort_unique(ctx, orc, n, k, hi):
    rng = np.random.default_rng(n * 10 + k)
    rows = rng.integers(-(hi // 2) if hi > 2 else 0, hi // 2 if hi > 2 else hi, (n, k), dtype=np.int64).astype(np.int32)
    vars_ = tuple(range(10, 10 + k))
    h = tb.tid_set_from_host(ctx, rows, vars_)
    got = _host(h)
    want = orc.TupleSet(vars_, orc.canonical(rows))
    _same(got, want)


# ---------------------------------------------------------------- K5/K6 joins

def _rand_set(orc, rng, vars_, n, hi, zeros=False):
    lo = 0 if zeros else 1
    return orc.TupleSet(tuple(vars_), orc.canonical(rng.integers(lo, hi, (n, len(vars_)))))


JOIN_SHAPES = [((0, 1), (0, 2)), ((0, 1), (2, 0)), ((1, 0), (2, 0)), ((0, 1, 2), (2, 1, 3)),
               ((0, 1), (0, 1, 2)), ((5, 6), (7, 8)), ((0,), (0,)), ((3, 0, 1), (1, 4, 0, 5))]


@pytest.mark.parametrize("algo", ["sort_merge", "hash"])
@pytest.mark.parametrize("shape", range(len(JOIN_SHAPES)))
@pytest.mark.parametrize("size", [(0, 10), (1, 1), (300, 500), (5000, 40_000), (30_000, 2000)])
def test_join_random_sets(ctx, orc, algo, shape, size):
    lv, rv = JOIN_SHAPES[shape]
    rng = np.random.default_rng(hash((shape, size)) % 2**32)
    nl, nr = size
    hi = 6 if (lv, rv) == ((5, 6), (7, 8)) else max(4, int(np.sqrt(max(nl, nr))) // 3)
    if (lv, rv) == ((5, 6), (7, 8)):  # cross product: keep it small
        nl, nr = min(nl, 300), min(nr, 200)
    L = _rand_set(orc, rng, lv, nl, hi, zeros=True)
    R = _rand_set(orc, rng, rv, nr, hi, zeros=True)
    hl = tb.tid_set_from_host(ctx, L.rows, lv)
    hr = tb.tid_set_from_host(ctx, R.rows, rv)
    j = tb.tid_join(ctx, hl, hr, algo)
    _same(_host(j), orc.join(L, R))
    tb.tid_set_free(hl)
    tb.tid_set_free(hr)


@pytest.mark.parametrize("shape", range(len(JOIN_SHAPES)))
@pytest.mark.parametrize("size", [(0, 10), (10, 0), (1, 1), (300, 500), (5000, 40_000), (30_000, 2000)])
def test_left_join_random_sets(ctx, orc, shape, size):
    """Left outer join (OPTIONAL) equals the oracle's, unmatched left rows padded with 0."""
    lv, rv = JOIN_SHAPES[shape]
    rng = np.random.default_rng((hash((shape, size)) + 17) % 2**32)
    nl, nr = size
    hi = 6 if (lv, rv) == ((5, 6), (7, 8)) else max(4, int(np.sqrt(max(nl, nr))) // 2)
    if (lv, rv) == ((5, 6), (7, 8)):
        nl, nr = min(nl, 300), min(nr, 200)
    L = _rand_set(orc, rng, lv, nl, hi, zeros=True)
    R = _rand_set(orc, rng, rv, nr, hi, zeros=True)
    hl = tb.tid_set_from_host(ctx, L.rows, lv)
    hr = tb.tid_set_from_host(ctx, R.rows, rv)
    _same(_host(tb.tid_join(ctx, hl, hr, "left")), orc.left_join(L, R))
    with pytest.raises(tb.TidError) as e:
        tb.tid_join(ctx, hl, hr, tb.TID_JOIN_LEFT | tb.JOIN["hash"])
    assert e.value.code == tb.TID_ERR_ARG
    tb.tid_set_free(hl)
    tb.tid_set_free(hr)


def test_optional_plans(ctx, orc):
    """Star plans on the university store with every join OPTIONAL: typed subjects
    with whichever properties they have."""
    st_np = synth.university_store(1_000_000)
    st = _store(ctx, st_np.s, st_np.p, st_np.o)
    for name, plan in synth.university_plans(st_np)[:16]:
        plan = [dict(nd, algo="left") if nd["op"] == "join" else nd for nd in plan]
        got = _host(tb.tid_exec(ctx, st, plan))
        want = orc.execute(st_np.s, st_np.p, st_np.o, plan)
        try:
            _same(got, want)
        except AssertionError as e:
            raise AssertionError(f"{name}: {e}")
    tb.tid_store_free(st)


def test_join_skewed_key(ctx, orc):
    """One key shared by many rows on both sides: its output spreads over threads."""
    rng = np.random.default_rng(3)
    L = orc.TupleSet((0, 1), orc.canonical(np.stack([np.r_[np.full(3000, 7), rng.integers(1, 50, 500)],
                                                     np.arange(3500)], 1)))
    R = orc.TupleSet((0, 2), orc.canonical(np.stack([np.r_[np.full(2000, 7), rng.integers(1, 50, 300)],
                                                     np.arange(2300)], 1)))
    hl = tb.tid_set_from_host(ctx, L.rows, (0, 1))
    hr = tb.tid_set_from_host(ctx, R.rows, (0, 2))
    want = orc.join(L, R, method="sortmerge")
    for algo in ("sort_merge", "hash"):
        _same(_host(tb.tid_join(ctx, hl, hr, algo)), want)
    tb.tid_set_free(hl)
    tb.tid_set_free(hr)


@pytest.mark.parametrize("kind", ["sparse", "fan_out"])
def test_join_output_partition(ctx, orc, kind):
    """The output rows are split over CTAs by probe rows and output rows
    together: long runs of probe rows without a match (sparse), and one key
    whose matches fill many CTAs' shares (fan-out), both against the oracle,
    inner and left, both algorithms."""
    rng = np.random.default_rng(17 if kind == "sparse" else 18)
    if kind == "sparse":  # 200K left keys, 40 of them present on the right
        lk = rng.choice(np.arange(1, 10_000_000), 200_000, replace=False)
        rk = np.r_[rng.choice(lk, 40, replace=False), rng.integers(10_000_001, 20_000_000, 1000)]
        L = orc.TupleSet((0, 1), orc.canonical(np.stack([lk, rng.integers(1, 9, lk.shape[0])], 1)))
        R = orc.TupleSet((0, 2), orc.canonical(np.stack([rk, np.arange(1, rk.shape[0] + 1)], 1)))
    else:  # key 5: 300 left rows x 2000 right rows = 600K output rows, among ordinary keys
        L = orc.TupleSet((0, 1), orc.canonical(np.stack([np.r_[np.full(300, 5), rng.integers(6, 40_000, 20_000)],
                                                         np.arange(1, 20_301)], 1)))
        R = orc.TupleSet((0, 2), orc.canonical(np.stack([np.r_[np.full(2000, 5), rng.integers(6, 40_000, 30_000)],
                                                         np.arange(1, 32_001)], 1)))
    hl = tb.tid_set_from_host(ctx, L.rows, (0, 1))
    hr = tb.tid_set_from_host(ctx, R.rows, (0, 2))
    want = orc.join(L, R, method="sortmerge")
    for algo in ("sort_merge", "hash"):
        _same(_host(tb.tid_join(ctx, hl, hr, algo)), want)
    want_left = orc.left_join(L, R)
    _same(_host(tb.tid_join(ctx, hl, hr, "left")), want_left)
    tb.tid_set_free(hl)
    tb.tid_set_free(hr)


def test_nine_relationship_types(ctx, orc):
    """Table 'Relationship between two triple patterns': OO, PP, SS, OP, OS, PS,
    PO, SP, SO -- the shared variable at each slot pairing -- on a small graph,
    equal to the solution-mapping brute force."""
    S, P, O = pins.tiny_graph(41, 60, ids=6)
    st = _store(ctx, S, P, O)
    X, Y, Z = 0, 1, 2
    for ia, ib in itertools.product(range(3), range(3)):
        va, vb = [-1, -1, -1], [-1, -1, -1]
        va[ia], vb[ib] = X, X
        va[(ia + 1) % 3], vb[(ib + 2) % 3] = Y, Z
        plan = [{"op": "match", "pattern": synth.Pattern(0, 0, 0, var=tuple(va))},
                {"op": "match", "pattern": synth.Pattern(0, 0, 0, var=tuple(vb))},
                {"op": "join", "inputs": [0, 1]}]
        for algo in ("sort_merge", "hash"):
            plan[2]["algo"] = algo
            vars_, rows = _host(tb.tid_exec(ctx, st, plan))
            want = pins.solutions(S, P, O, [((0, 0, 0), tuple(va)), ((0, 0, 0), tuple(vb))], vars_)
            assert rows.tolist() == [list(w) for w in want], ("SPO"[ia] + "SPO"[ib], algo)
    tb.tid_store_free(st)


# ---------------------------------------------------------------- K7 union / project

def test_union_and_project(ctx, orc):
    rng = np.random.default_rng(8)
    A = _rand_set(orc, rng, (0, 1), 5000, 40)
    B = _rand_set(orc, rng, (1, 2), 3000, 40)
    C = _rand_set(orc, rng, (0, 1), 5000, 40)
    D = _rand_set(orc, rng, (2,), 100, 400)
    hs = [tb.tid_set_from_host(ctx, t.rows, t.vars) for t in (A, B, C, D)]
    for combo in ([0], [0, 2], [0, 1], [2, 0, 1], [0, 1, 2, 3], [0, 0]):
        u = tb.tid_union(ctx, [hs[i] for i in combo])
        _same(_host(u), orc.union([(A, B, C, D)[i] for i in combo]))
    for vs in ((1,), (1, 0), (0, 1)):
        _same(_host(tb.tid_project(ctx, hs[0], vs)), orc.project(A, vs))
    for h in hs:
        tb.tid_set_free(h)


def test_errors_are_reported(ctx):
    h = tb.tid_set_from_host(ctx, np.array([[1, 2]], np.int32), (0, 1))
    with pytest.raises(tb.TidError) as e:
        tb.tid_filter(ctx, h, [(9, "eq", 1)])
    assert e.value.code == tb.TID_ERR_ARG
    with pytest.raises(tb.TidError):
        tb.tid_project(ctx, h, (0, 0))
    with pytest.raises(tb.TidError):
        tb.tid_join(ctx, h, h, 7)
    tb.tid_set_free(h)


# ---------------------------------------------------------------- plans

def test_worked_example_plan(ctx):
    g = json.load(open(os.path.join(GOLDEN, "rule11_worked_example.json")))
    a = np.array(g["store"], np.int32)
    st = _store(ctx, a[:, 0], a[:, 1], a[:, 2])
    X, Y, Z = 0, 1, 2
    for algo in ("sort_merge", "hash"):
        plan = [{"op": "match", "pattern": synth.Pattern(0, 84, 0, var=(X, -1, Y))},
                {"op": "match", "pattern": synth.Pattern(0, 84, 0, var=(Y, -1, Z))},
                {"op": "join", "inputs": [0, 1], "algo": algo},
                {"op": "project", "input": 2, "vars": [X, Z]}]
        vars_, rows = _host(tb.tid_exec(ctx, st, plan))
        assert vars_ == (X, Z)
        assert sorted(map(tuple, rows.tolist())) == sorted(map(tuple, g["result_xz"]))
    tb.tid_store_free(st)


@pytest.mark.parametrize("algo", ["auto", "sort_merge", "hash"])
def test_university_plans(ctx, orc, algo):
    st_np = synth.university_store(1_000_000)
    st = _store(ctx, st_np.s, st_np.p, st_np.o)
    for name, plan in synth.university_plans(st_np):
        plan = [dict(nd, algo=algo) if nd["op"] == "join" else nd for nd in plan]
        got = _host(tb.tid_exec(ctx, st, plan))
        want = orc.execute(st_np.s, st_np.p, st_np.o, plan)
        try:
            _same(got, want)
        except AssertionError as e:
            raise AssertionError(f"{name}: {e}")
    tb.tid_store_free(st)
