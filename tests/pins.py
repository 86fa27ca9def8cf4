"""Pins for the CPU oracle: facts fixed by the paper or by mathematics, computed
WITHOUT the oracle's own formulas.

* the worked example the paper prints (Rule 11, golden file);
* solution-mapping brute force: a pattern's answers are the substitutions of
  its variables, drawn from the store's domain, whose instantiated triple is in
  the graph -- a different statement of "matches" than the oracle's per-slot
  wildcard test, and the one that also defines joins of several patterns;
* value tallies (np.bincount / sort-based counts) for single- and two-bound
  patterns, and the total N for (?,?,?);
* algebraic laws of union, filter and join (cross product then selection).

Each pin raises AssertionError when the oracle disagrees.  ``ALL_PINS`` is run
both against the real oracle and against mutated copies of it, which must fail.
"""
from __future__ import annotations

import itertools
import json
import os
from collections import Counter

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------------------
# solution-mapping brute force (independent of the oracle)
# ---------------------------------------------------------------------------

def tiny_graph(seed, n, ids=8):
    """A random set of <= n triples over IDs 1..ids, in random order."""
    rng = np.random.default_rng(seed)
    t = rng.integers(1, ids + 1, size=(n, 3))
    seen, rows = set(), []
    for r in map(tuple, t.tolist()):
        if r not in seen:
            seen.add(r)
            rows.append(r)
    a = np.array(rows, dtype=np.int32).reshape(-1, 3)
    return a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy()


def _slots(key, var, fresh):
    """Slot terms: ('c', id) for a constant, ('v', name) for a variable."""
    out = []
    for j in range(3):
        if int(key[j]) != 0:
            out.append(("c", int(key[j])))
        elif int(var[j]) >= 0:
            out.append(("v", ("named", int(var[j]))))
        else:
            out.append(("v", ("anon", next(fresh))))
    return out


def solutions(S, P, O, patterns, project_vars):
    """Distinct projections of the substitutions (over the graph's domain) under
    which every pattern instantiates to a stored triple."""
    G = set(zip(S.tolist(), P.tolist(), O.tolist()))
    dom = sorted(set(S.tolist()) | set(P.tolist()) | set(O.tolist()))
    fresh = itertools.count()
    slotted = [_slots(k, v, fresh) for k, v in patterns]
    names = []
    for sl in slotted:
        for kind, x in sl:
            if kind == "v" and x not in names:
                names.append(x)
    out = set()
    for theta in itertools.product(dom, repeat=len(names)):
        env = dict(zip(names, theta))
        if all(tuple(x if kind == "c" else env[x] for kind, x in sl) in G for sl in slotted):
            out.add(tuple(env[("named", v)] for v in project_vars))
    return sorted(out)


def positions(S, P, O, key):
    """Positions of the stored triples that are instances of the key (0 = "?"),
    by enumerating substitutions of the "?" slots."""
    index = {t: i for i, t in enumerate(zip(S.tolist(), P.tolist(), O.tolist()))}
    dom = sorted(set(S.tolist()) | set(P.tolist()) | set(O.tolist()))
    free = [j for j in range(3) if int(key[j]) == 0]
    hits = []
    for theta in itertools.product(dom, repeat=len(free)):
        t = [int(x) for x in key]
        for j, v in zip(free, theta):
            t[j] = v
        i = index.get(tuple(t))
        if i is not None:
            hits.append(i)
    return sorted(hits)


# ---------------------------------------------------------------------------
# pins
# ---------------------------------------------------------------------------

def pin_golden_rule11(o):
    """Section 5, Rule (11) worked example: values printed in the paper."""
    g = json.load(open(os.path.join(GOLDEN, "rule11_worked_example.json")))
    st = np.array(g["store"], np.int32)
    S, P, O = st[:, 0].copy(), st[:, 1].copy(), st[:, 2].copy()
    n = len(st)
    idx = o.match(S, P, O, g["step1"]["key"])
    flags = np.zeros(n, int)
    flags[idx] = 1
    assert flags.tolist() == g["step1"]["flags"], (flags, g["step1"])
    lists = o.match_multi(S, P, O, g["step2"]["keys"])
    flags2 = np.zeros(n, int)
    for lst in lists:
        flags2[lst] = 1
    assert flags2.tolist() == g["step2"]["flags"], (flags2, g["step2"])
    # x subClassOf y . y subClassOf z  -> (x, z)
    X, Y, Z = 0, 1, 2
    a = o.bind(S, P, O, (0, 84, 0), (X, -1, Y), o.match(S, P, O, (0, 84, 0)))
    b = o.bind(S, P, O, (0, 84, 0), (Y, -1, Z), o.match(S, P, O, (0, 84, 0)))
    r = o.project(o.join(a, b), (X, Z))
    assert r.vars == (X, Z)
    assert sorted(map(tuple, r.rows.tolist())) == sorted(map(tuple, g["result_xz"])), r.rows


def pin_match_bruteforce(o):
    """Every key in {0..8}^3 on small random graphs: positions equal the
    substitution-enumeration answer."""
    for seed, n in ((1, 40), (2, 64), (3, 7)):
        S, P, O = tiny_graph(seed, n)
        for key in itertools.product(range(9), repeat=3):
            got = o.match(S, P, O, key).tolist()
            assert got == positions(S, P, O, key), (seed, key)
    S, P, O = (np.zeros(0, np.int32),) * 3
    assert o.match(S, P, O, (0, 0, 0)).tolist() == []


def pin_match_tallies(o):
    """Counts equal value tallies: count(s,?,?) = occurrences of s in S (and for
    p, o); count(s,p,?) = occurrences of the pair; count(?,?,?) = N."""
    rng = np.random.default_rng(7)
    n = 20000
    S = rng.integers(1, 300, n).astype(np.int32)
    P = rng.integers(1, 12, n).astype(np.int32)
    O = rng.integers(1, 500, n).astype(np.int32)
    assert o.match(S, P, O, (0, 0, 0)).shape[0] == n
    for col, pos in ((S, 0), (P, 1), (O, 2)):
        h = np.bincount(col)
        for v in rng.choice(np.unique(col), 10, replace=False):
            key = [0, 0, 0]
            key[pos] = int(v)
            assert o.match(S, P, O, key).shape[0] == h[v], (pos, v)
    pair = Counter(zip(S.tolist(), P.tolist()))
    for (s, p) in list(pair)[:40]:
        assert o.match(S, P, O, (s, p, 0)).shape[0] == pair[(s, p)]
    pairo = Counter(zip(P.tolist(), O.tolist()))
    for (p, oo) in list(pairo)[:40]:
        assert o.match(S, P, O, (0, p, oo)).shape[0] == pairo[(p, oo)]
    tot = sum(o.match(S, P, O, (0, int(p), 0)).shape[0] for p in np.unique(P))
    assert tot == n
    # multi-key lists equal the single-key lists (one pass vs many)
    keys = [(0, 3, 0), (5, 0, 0), (0, 0, 7), (0, 3, 0), (5, 3, 0)]
    multi = o.match_multi(S, P, O, keys)
    for k, lst in zip(keys, multi):
        assert lst.shape[0] == o.match(S, P, O, k).shape[0]


def pin_bind_join_bruteforce(o):
    """Two-pattern conjunctions in all nine relationship types of the paper's
    table (shared variable at S/P/O on either side), plus repeated variables:
    bind + join + project equals the solution-mapping enumeration."""
    X, Y, Z, W = 0, 1, 2, 3
    # (pattern A, pattern B) with keys drawn per case; slot of the shared var varies
    shapes = []
    for ia in range(3):
        for ib in range(3):
            va, vb = [-1, -1, -1], [-1, -1, -1]
            va[ia] = X
            vb[ib] = X
            va[(ia + 1) % 3] = Y
            vb[(ib + 2) % 3] = Z
            shapes.append((tuple(va), tuple(vb)))
    shapes.append(((X, -1, X), (X, -1, Y)))          # repeated variable
    shapes.append(((X, Y, -1), (X, Y, Z)))           # two shared variables
    shapes.append(((X, -1, Y), (W, -1, Z)))          # no shared variable: cross product
    for seed in (11, 12):
        S, P, O = tiny_graph(seed, 30, ids=5)
        rng = np.random.default_rng(seed)
        for va, vb in shapes:
            ka = tuple(0 if va[j] >= 0 else int(rng.integers(1, 6)) for j in range(3))
            kb = tuple(0 if vb[j] >= 0 else int(rng.integers(1, 6)) for j in range(3))
            # keep some cases all-variable in the unconstrained slot
            a = o.bind(S, P, O, ka, va, o.match(S, P, O, ka))
            b = o.bind(S, P, O, kb, vb, o.match(S, P, O, kb))
            # a result vector has one column per distinct variable, in slot order
            assert a.vars == tuple(dict.fromkeys(v for v in va if v >= 0)), (va, a.vars)
            assert b.vars == tuple(dict.fromkeys(v for v in vb if v >= 0)), (vb, b.vars)
            j = o.join(a, b)
            assert j.vars == a.vars + tuple(v for v in b.vars if v not in a.vars), (a.vars, b.vars, j.vars)
            want = solutions(S, P, O, [(ka, va), (kb, vb)], j.vars)
            assert sorted(map(tuple, j.rows.tolist())) == want, (seed, va, vb, ka, kb)
            assert j.rows.tolist() == [list(r) for r in want]  # canonical order
            # |join| = sum over keys of cntL * cntR (no zero keys here)
            sh = [v for v in a.vars if v in b.vars]
            ca = Counter(tuple(r[a.vars.index(v)] for v in sh) for r in a.rows.tolist())
            cb = Counter(tuple(r[b.vars.index(v)] for v in sh) for r in b.rows.tolist())
            assert j.n == sum(ca[k] * cb.get(k, 0) for k in ca)


def pin_bind_anonymous_wildcards(o):
    """A result vector keeps one row per distinct value of its named variables:
    an anonymous "?" is existential (the solution mappings projected on the named
    variables), and a variable named twice needs equal terms."""
    X, Y = 0, 1
    cases = [((0, 0, 0), (X, -1, -1)), ((0, 0, 0), (-1, X, -1)), ((0, 0, 0), (-1, -1, X)),
             ((0, 3, 0), (X, -1, -1)), ((0, 0, 0), (X, -1, Y)), ((0, 0, 2), (X, Y, -1)),
             ((0, 0, 0), (X, -1, X)), ((1, 0, 0), (-1, X, -1))]
    for seed in (41, 42):
        S, P, O = tiny_graph(seed, 45, ids=5)
        for key, var in cases:
            got = o.bind(S, P, O, key, var, o.match(S, P, O, key))
            named = tuple(dict.fromkeys(v for v in var if v >= 0))
            assert got.vars == named, (key, var)
            assert got.rows.tolist() == [list(w) for w in solutions(S, P, O, [(key, var)], named)], (seed, key, var)


def pin_join_cross_product(o):
    """join(L, R) = rows of L x R whose shared columns agree (and are bound)."""
    rng = np.random.default_rng(5)
    for trial in range(30):
        kl, kr = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        lv = tuple(rng.choice(6, kl, replace=False).tolist())
        rv = tuple(rng.choice(6, kr, replace=False).tolist())
        L = o.TupleSet(lv, o.canonical(rng.integers(0, 4, (int(rng.integers(0, 25)), kl))))
        R = o.TupleSet(rv, o.canonical(rng.integers(0, 4, (int(rng.integers(0, 25)), kr))))
        j = o.join(L, R)
        sh = [v for v in lv if v in rv]
        want = set()
        for l in L.rows.tolist():
            for r in R.rows.tolist():
                if all(l[lv.index(v)] == r[rv.index(v)] and l[lv.index(v)] != 0 for v in sh):
                    want.add(tuple(l) + tuple(r[i] for i, v in enumerate(rv) if v not in lv))
        assert j.rows.tolist() == [list(x) for x in sorted(want)], trial
        js = o.join(L, R, method="sortmerge")
        assert np.array_equal(js.rows, j.rows)


def pin_union_laws(o):
    """Union is commutative and idempotent, pads missing variables with 0, and
    equals the Python set union of padded rows."""
    rng = np.random.default_rng(9)
    A = o.TupleSet((0, 1), o.canonical(rng.integers(1, 5, (30, 2))))
    B = o.TupleSet((1, 2), o.canonical(rng.integers(1, 5, (30, 2))))
    C = o.TupleSet((0, 1), o.canonical(rng.integers(1, 5, (30, 2))))
    u = o.union([A, C])
    assert np.array_equal(u.rows, o.union([C, A]).rows)
    assert np.array_equal(o.union([A, A]).rows, A.rows)
    assert np.array_equal(o.union([u, A]).rows, u.rows)
    want = sorted(set(map(tuple, A.rows.tolist())) | set(map(tuple, C.rows.tolist())))
    assert u.rows.tolist() == [list(x) for x in want]
    ab = o.union([A, B])
    assert ab.vars == (0, 1, 2)
    want = sorted({(a, b, 0) for a, b in A.rows.tolist()} | {(0, b, c) for b, c in B.rows.tolist()})
    assert ab.rows.tolist() == [list(x) for x in want]


def pin_filter_algebra(o):
    """Full range is the identity on bound rows; ranges compose by
    intersection; EQ/NE split the bound rows; LT/LE/GT/GE are ranges; a row
    whose value is 0 (unbound) never passes."""
    rng = np.random.default_rng(4)
    T = o.TupleSet((3, 4), o.canonical(rng.integers(0, 50, (400, 2))))
    col = T.rows[:, 1]
    bound = T.rows[col != 0]
    full = o.filter(T, 4, "range", 1, 2 ** 31 - 1)
    assert np.array_equal(full.rows, bound)
    for a, b, c, d in ((3, 30, 10, 40), (0, 49, 20, 20), (5, 9, 12, 15)):
        two = o.filter(o.filter(T, 4, "range", a, b), 4, "range", c, d)
        one = o.filter(T, 4, "range", max(a, c), min(b, d))
        assert np.array_equal(two.rows, one.rows)
    for v in (0, 1, 17, 49):
        eq = o.filter(T, 4, "eq", v)
        ne = o.filter(T, 4, "ne", v)
        assert eq.n + ne.n == bound.shape[0]
        assert np.array_equal(eq.rows, o.filter(T, 4, "range", v, v).rows)
        assert np.array_equal(o.filter(T, 4, "lt", v).rows, o.filter(T, 4, "range", -2 ** 31, v - 1).rows)
        assert np.array_equal(o.filter(T, 4, "le", v).rows, o.filter(T, 4, "range", -2 ** 31, v).rows)
        assert np.array_equal(o.filter(T, 4, "gt", v).rows, o.filter(T, 4, "range", v + 1, 2 ** 31 - 1).rows)
        assert np.array_equal(o.filter(T, 4, "ge", v).rows, o.filter(T, 4, "range", v, 2 ** 31 - 1).rows)
        assert (o.filter(T, 4, "ge", v).rows[:, 1] >= max(v, 1)).all()
    # numbers counted directly
    assert o.filter(T, 4, "range", 10, 20).n == int(((col >= 10) & (col <= 20)).sum())


def pin_canonical(o):
    """Canonical form = Python's sorted set of row tuples."""
    rng = np.random.default_rng(3)
    for k in (1, 2, 3, 5, 8):
        rows = rng.integers(-3, 6, (300, k))
        got = o.canonical(rows)
        want = sorted(set(map(tuple, rows.tolist())))
        assert got.tolist() == [list(x) for x in want], k


def pin_project(o):
    """SELECT keeps the named variables in the named order, with DISTINCT: the
    Python set of the picked tuple entries (columns drawn from disjoint value
    ranges, so a swapped or re-sorted column list cannot pass)."""
    rng = np.random.default_rng(6)
    rows = np.stack([rng.integers(1, 6, 200), rng.integers(10, 14, 200), rng.integers(20, 60, 200)], axis=1)
    T = o.TupleSet((0, 1, 2), o.canonical(rows))
    for pick in ((2, 0), (1,), (2, 1, 0), (0, 2)):
        pr = o.project(T, pick)
        want = sorted({tuple(r[v] for v in pick) for r in T.rows.tolist()})
        assert pr.vars == pick and pr.rows.tolist() == [list(x) for x in want], pick


def pin_left_join_rowwise(o):
    """Left join, row by row: each left row with its matching right rows (all
    shared columns equal and bound), or alone with the right side's other columns
    0 when it has none."""
    rng = np.random.default_rng(31)
    for t in range(30):
        kl, kr = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        lv = tuple(int(x) for x in rng.choice(6, size=kl, replace=False))
        rv = tuple(int(x) for x in rng.choice(6, size=kr, replace=False))
        L = o.TupleSet(lv, o.canonical(rng.integers(0, 4, (int(rng.integers(0, 40)), kl)).astype(np.int32)))
        R = o.TupleSet(rv, o.canonical(rng.integers(0, 4, (int(rng.integers(0, 40)), kr)).astype(np.int32)))
        shared = [v for v in lv if v in rv]
        rest = [j for j, v in enumerate(rv) if v not in lv]
        want = set()
        for l in L.rows.tolist():
            hits = [r for r in R.rows.tolist()
                    if all(l[lv.index(v)] == r[rv.index(v)] != 0 for v in shared)]
            if hits:
                for r in hits:
                    want.add(tuple(l) + tuple(r[j] for j in rest))
            else:
                want.add(tuple(l) + (0,) * len(rest))
        got = o.left_join(L, R)
        assert got.vars == lv + tuple(rv[j] for j in rest)
        assert got.rows.tolist() == [list(x) for x in sorted(want)], t


def pin_outer_joins_rowwise(o):
    """Right and full outer joins, row by row: every pair of rows whose shared
    columns are all equal and bound gives a row; a right row with no such pair
    appears alone with the left side's other columns 0 (right and full), and so
    does a left row with no pair, with the right side's other columns 0 (full).
    Columns as the inner join's: the left's, then the right's others."""
    rng = np.random.default_rng(37)
    for t in range(30):
        kl, kr = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        lv = tuple(int(x) for x in rng.choice(6, size=kl, replace=False))
        rv = tuple(int(x) for x in rng.choice(6, size=kr, replace=False))
        L = o.TupleSet(lv, o.canonical(rng.integers(0, 4, (int(rng.integers(0, 40)), kl)).astype(np.int32)))
        R = o.TupleSet(rv, o.canonical(rng.integers(0, 4, (int(rng.integers(0, 40)), kr)).astype(np.int32)))
        shared = [v for v in lv if v in rv]
        rest = [j for j, v in enumerate(rv) if v not in lv]
        out_vars = lv + tuple(rv[j] for j in rest)

        def pairs(l, r):
            return all(l[lv.index(v)] == r[rv.index(v)] != 0 for v in shared)
        inner, lonely_l, lonely_r = set(), set(), set()
        for l in L.rows.tolist():
            if not any(pairs(l, r) for r in R.rows.tolist()):
                lonely_l.add(tuple(l) + (0,) * len(rest))
            for r in R.rows.tolist():
                if pairs(l, r):
                    inner.add(tuple(l) + tuple(r[j] for j in rest))
        for r in R.rows.tolist():
            if not any(pairs(l, r) for l in L.rows.tolist()):
                lonely_r.add(tuple(r[rv.index(v)] if v in rv else 0 for v in out_vars))
        got_r, got_f = o.right_join(L, R), o.full_join(L, R)
        assert got_r.vars == out_vars and got_f.vars == out_vars
        assert got_r.rows.tolist() == [list(x) for x in sorted(inner | lonely_r)], t
        assert got_f.rows.tolist() == [list(x) for x in sorted(inner | lonely_l | lonely_r)], t


# RDFS rules of the paper's entailment table (Section 5), for the brute force:
# two premises and a conclusion over variable names and vocabulary terms
_RULES_BF = {
    2: ((("p", "domain", "D"), ("s", "p", "o")), ("s", "type", "D")),
    3: ((("p", "range", "R"), ("s", "p", "o")), ("o", "type", "R")),
    5: ((("p", "subprop", "q"), ("q", "subprop", "r")), ("p", "subprop", "r")),
    7: ((("p", "subprop", "q"), ("s", "p", "o")), ("s", "q", "o")),
    9: ((("x", "subclass", "y"), ("s", "type", "x")), ("s", "type", "y")),
    11: ((("x", "subclass", "y"), ("y", "subclass", "z")), ("x", "subclass", "z")),
}


def _unify(tpl, triple, env, vocab):
    env = dict(env)
    for term, val in zip(tpl, triple):
        if term in vocab:
            if vocab[term] != val:
                return None
        elif term in env:
            if env[term] != val:
                return None
        else:
            env[term] = val
    return env


def entail_bruteforce(S, P, O, rule, vocab):
    """Conclusions of a rule by trying every ordered pair of stored triples as
    (premise 1, premise 2) instances."""
    G = list(zip(S.tolist(), P.tolist(), O.tolist()))
    (t1, t2), then = _RULES_BF[rule]
    out = set()
    for a in G:
        e1 = _unify(t1, a, {}, vocab)
        if e1 is None:
            continue
        for b in G:
            e2 = _unify(t2, b, e1, vocab)
            if e2 is not None:
                out.add(tuple(vocab[t] if t in vocab else e2[t] for t in then))
    return sorted(out)


def pin_entail_golden(o):
    """Section 5, Rule (11) walk-through through the rule evaluator: 4 schema
    matches, 3 distinct terms (the three keys of the second search), 2 matches of
    the second search, 2 conclusions (76, 84, 78) and (76, 84, 77)."""
    g = json.load(open(os.path.join(GOLDEN, "rule11_worked_example.json")))
    st = np.array(g["store"], np.int32)
    vocab = {"type": 1, "domain": 2, "range": 3, "subprop": 4, "subclass": 84}
    out, stats = o.entail(st[:, 0].copy(), st[:, 1].copy(), st[:, 2].copy(), 11, vocab)
    assert out.vars == (0, 1, 2)
    assert sorted(map(tuple, out.rows.tolist())) == sorted((x, 84, z) for x, z in g["result_xz"])
    assert stats["res1"] == sum(g["step1"]["flags"]) and stats["dist1"] == len(g["step2"]["keys"])
    assert stats["res2"] == sum(g["step2"]["flags"]) and stats["all"] == len(g["result_xz"])


def pin_entail_bruteforce(o):
    """Every rule on small random graphs whose IDs include the vocabulary terms:
    the conclusions equal the pairwise brute force."""
    vocab = {"type": 1, "domain": 2, "range": 3, "subprop": 4, "subclass": 5}
    for seed in range(6):
        S, P, O = tiny_graph(100 + seed, 90, ids=7)
        for rule in _RULES_BF:
            out, stats = o.entail(S, P, O, rule, vocab)
            want = entail_bruteforce(S, P, O, rule, vocab)
            assert out.rows.tolist() == [list(t) for t in want], (seed, rule)
            assert stats["all"] == len(want)


def pin_execute_plans(o):
    """Whole plans (star, chain, union, filter, project) on small graphs equal
    the solution-mapping enumeration of the same graph pattern (the plan nodes
    of Sections 4.1-4.3 evaluated in order)."""
    from paper_1807_01409_gb300.synth import Pattern
    X, Y, Z = 0, 1, 2
    S, P, O = tiny_graph(31, 40, ids=6)
    star = [{"op": "match", "pattern": Pattern(0, 2, 0, var=(X, -1, Y))},
            {"op": "match", "pattern": Pattern(0, 3, 0, var=(X, -1, Z))},
            {"op": "join", "inputs": [0, 1]}]
    r = o.execute(S, P, O, star)
    want = solutions(S, P, O, [((0, 2, 0), (X, -1, Y)), ((0, 3, 0), (X, -1, Z))], r.vars)
    assert r.rows.tolist() == [list(w) for w in want]
    chain = [{"op": "match", "pattern": Pattern(0, 0, 0, var=(X, -1, Y))},
             {"op": "match", "pattern": Pattern(0, 4, 0, var=(Y, -1, Z))},
             {"op": "join", "inputs": [0, 1]},
             {"op": "project", "input": 2, "vars": [X, Z]}]
    r = o.execute(S, P, O, chain)
    want = solutions(S, P, O, [((0, 0, 0), (X, -1, Y)), ((0, 4, 0), (Y, -1, Z))], (X, Z))
    assert r.rows.tolist() == [list(w) for w in want]
    # FILTER (?Y in [2, 4]) over the chain's first pattern
    flt = [{"op": "match", "pattern": Pattern(0, 0, 0, var=(X, -1, Y))},
           {"op": "filter", "input": 0, "var": Y, "cmp": "range", "a": 2, "b": 4}]
    r = o.execute(S, P, O, flt)
    want = [w for w in solutions(S, P, O, [((0, 0, 0), (X, -1, Y))], (X, Y)) if 2 <= w[1] <= 4]
    assert r.rows.tolist() == [list(w) for w in want]
    # UNION of two branches with different variables
    un = [{"op": "match", "pattern": Pattern(1, 0, 0, var=(-1, X, Y))},
          {"op": "match", "pattern": Pattern(0, 2, 0, var=(Y, -1, Z))},
          {"op": "union", "inputs": [0, 1]}]
    r = o.execute(S, P, O, un)
    a = solutions(S, P, O, [((1, 0, 0), (-1, X, Y))], (X, Y))
    b = solutions(S, P, O, [((0, 2, 0), (Y, -1, Z))], (Y, Z))
    want = sorted({(x, y, 0) for x, y in a} | {(0, y, z) for y, z in b})
    assert r.vars == (X, Y, Z) and r.rows.tolist() == [list(w) for w in want]
    # a chain joined as OPTIONAL (left), right and full outer joins
    a = solutions(S, P, O, [((0, 2, 0), (X, -1, Y))], (X, Y))
    b = solutions(S, P, O, [((0, 3, 0), (Y, -1, Z))], (Y, Z))
    inner = {(x, y, z) for x, y in a for y2, z in b if y == y2}
    only_a = {(x, y, 0) for x, y in a if not any(y == y2 for y2, _ in b)}
    only_b = {(0, y, z) for y, z in b if not any(y == y1 for _, y1 in a)}
    for kind, want in (("left", inner | only_a), ("right", inner | only_b), ("full", inner | only_a | only_b)):
        plan = [{"op": "match", "pattern": Pattern(0, 2, 0, var=(X, -1, Y))},
                {"op": "match", "pattern": Pattern(0, 3, 0, var=(Y, -1, Z))},
                {"op": "join", "inputs": [0, 1], "algo": kind}]
        r = o.execute(S, P, O, plan)
        assert r.vars == (X, Y, Z) and r.rows.tolist() == [list(w) for w in sorted(want)], kind


ALL_PINS = [pin_golden_rule11, pin_match_bruteforce, pin_match_tallies,
            pin_bind_join_bruteforce, pin_bind_anonymous_wildcards, pin_join_cross_product, pin_union_laws,
            pin_filter_algebra, pin_canonical, pin_project, pin_entail_golden,
            pin_entail_bruteforce, pin_left_join_rowwise, pin_outer_joins_rowwise, pin_execute_plans]
