"""Edge cases of the search and the operators through the C ABI against the
CPU oracle, bit-exact: IDs at both ends of the positive int32 range (single
and batched search over every key, plans whose sort keys span 31 bits per
column) and store shards (Section 3's per-GPU chunks) as borrowed views of one
store.  Collected after the other operator files."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1807_01409_gb300 import binding as tb
from paper_1807_01409_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1807_01409_gb300 import build
    build.build()
    c = tb.tid_ctx_create(0, None)
    yield c
    tb.tid_ctx_destroy(c)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def _store(ctx, S, P, O):
    return tb.tid_load(ctx, _dev(S), _dev(P), _dev(O), copy=1)


def _match(ctx, store, key):
    h = tb.tid_match(ctx, store, key)
    try:
        return tb.tid_set_to_host(h)[:, 0].copy()
    finally:
        tb.tid_set_free(h)


def _lists(handles):
    out = []
    for h in handles:
        out.append(tb.tid_set_to_host(h)[:, 0].copy())
        tb.tid_set_free(h)
    return out


def _host(h):
    try:
        return tb.tid_set_info(h)["vars"], tb.tid_set_to_host(h).copy()
    finally:
        tb.tid_set_free(h)


def _same(got, want):
    gv, gr = got
    assert tuple(gv) == tuple(want.vars), (gv, want.vars)
    assert gr.shape == want.rows.shape, (gr.shape, want.rows.shape)
    assert np.array_equal(gr, want.rows)


@pytest.mark.parametrize("world", [2, 3])
def test_shards_concatenate_to_the_whole_store(ctx, orc, world):
    """Section 3's per-GPU chunks: each shard is a borrowed view of a contiguous
    range; its local lists offset by the shard's base and concatenated in rank
    order equal the whole store's list."""
    from paper_1807_01409_gb300 import shard
    st = synth.university_store(200_003)
    cols = [_dev(c) for c in (st.s, st.p, st.o)]
    stores = [shard.load_shard(ctx, *cols, world, r) for r in range(world)]
    try:
        for pat, _, _ in synth.university_queries(st)[:12]:
            key = pat.key()
            got = np.concatenate([shard.global_indices(_match(ctx, sh, key), base) for sh, base in stores])
            assert np.array_equal(got, orc.match(st.s, st.p, st.o, key)), key
    finally:
        for sh, _ in stores:
            tb.tid_store_free(sh)


EXTREME = np.array([1, 2, 3, 2 ** 30 - 1, 2 ** 30, 2 ** 30 + 1, 2 ** 31 - 2, 2 ** 31 - 1], np.int32)


def test_match_extreme_ids(ctx, orc):
    """IDs at both ends of the positive int32 range (entities just below the
    literal base 2^30, literals above it, the largest ID)."""
    rng = np.random.default_rng(77)
    n = 300_001
    S, P, O = (EXTREME[rng.integers(0, EXTREME.size, n)] for _ in range(3))
    store = tb.tid_load(ctx, _dev(S), _dev(P), _dev(O), copy=1)
    vals = [0] + EXTREME.tolist()
    for key in [(a, b, c) for a in vals[::3] for b in vals[::2] for c in vals[::3]]:
        assert np.array_equal(_match(ctx, store, key), orc.match(S, P, O, key)), key
    tb.tid_store_free(store)


def test_batch_extreme_ids(ctx, orc):
    """Every key over IDs at both ends of the positive int32 range, including
    the largest, as one batch."""
    ext = np.array([1, 2, 2 ** 30 - 1, 2 ** 30, 2 ** 31 - 2, 2 ** 31 - 1], np.int32)
    rng = np.random.default_rng(78)
    n = 200_003
    S, P, O = (ext[rng.integers(0, ext.size, n)] for _ in range(3))
    store = tb.tid_load(ctx, _dev(S), _dev(P), _dev(O), copy=1)
    vals = [0] + ext.tolist()
    keys = [(a, b, c) for a in vals for b in vals for c in vals]
    got = _lists(tb.tid_match_batch(ctx, store, keys))
    for k, g in zip(keys, got):
        assert np.array_equal(g, orc.match(S, P, O, k)), k
    tb.tid_store_free(store)


@pytest.mark.parametrize("algo", ["sort_merge", "hash"])
def test_extreme_id_plans(ctx, orc, algo):
    """Plans over IDs at both ends of the positive int32 range: packed sort keys
    of 31 bits per column (two columns in 64 bits, three past it), joins, a
    union, a literal-range filter and a projection."""
    vals = np.r_[np.arange(1, 17), np.arange(2 ** 30 - 16, 2 ** 30 + 16), np.arange(2 ** 31 - 16, 2 ** 31)]
    vals = vals.astype(np.int64)
    rng = np.random.default_rng(79)
    t = np.unique(np.stack([rng.choice(vals, 60_000) for _ in range(3)], axis=1), axis=0)
    t = t[rng.permutation(t.shape[0])].astype(np.int32)
    S, P, O = t[:, 0].copy(), t[:, 1].copy(), t[:, 2].copy()
    st = _store(ctx, S, P, O)
    p1, p2 = int(vals[0]), int(vals[-1])
    X, Y, Z, Q = 0, 1, 2, 3
    plans = [
        [{"op": "match", "pattern": synth.Pattern(0, p1, 0, var=(X, -1, Y))},
         {"op": "match", "pattern": synth.Pattern(0, p2, 0, var=(Y, -1, Z))},
         {"op": "join", "inputs": [0, 1], "algo": algo},
         {"op": "project", "input": 2, "vars": [Z, X]}],
        [{"op": "match", "pattern": synth.Pattern(0, 0, 0, var=(X, Q, Y))},
         {"op": "match", "pattern": synth.Pattern(0, p2, 0, var=(Y, -1, Z))},
         {"op": "join", "inputs": [0, 1], "algo": algo}],
        [{"op": "match", "pattern": synth.Pattern(0, p1, 0, var=(X, -1, Y))},
         {"op": "match", "pattern": synth.Pattern(0, p2, 0, var=(X, -1, Z))},
         {"op": "union", "inputs": [0, 1]},
         {"op": "filter", "input": 2, "var": X, "cmp": "range", "a": 2 ** 30, "b": 2 ** 31 - 1}],
    ]
    for plan in plans:
        _same(_host(tb.tid_exec(ctx, st, plan)), orc.execute(S, P, O, plan))
    tb.tid_store_free(st)


def test_bounded_wait_gives_up_and_the_context_recovers(ctx, orc):
    """Failure detection without a GPU fault: a wait that nothing will end (a
    barrier no other CTA reaches) gives up after its poll limit, the context
    reports TID_ERR_TIMEOUT once, and then answers correctly."""
    import time
    t0 = time.perf_counter()
    assert tb.tid_ctx_test_bounded_wait(ctx, 2000) == tb.TID_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60
    tb.tid_ctx_sync(ctx)  # reported once, then clear
    with pytest.raises(tb.TidError) as e:
        tb._check(tb.lib().tid_ctx_test_bounded_wait(ctx, 0), "polls")
    assert e.value.code == tb.TID_ERR_ARG
    st = synth.tiny_store(20_000)
    store = tb.tid_load(ctx, _dev(st.s), _dev(st.p), _dev(st.o), copy=1)
    for q in synth.tiny_queries(st)[:6]:
        assert np.array_equal(_match(ctx, store, q.key()), orc.match(st.s, st.p, st.o, q.key()))
    tb.tid_store_free(store)


OUTER_SHAPES = [((0, 1), (0, 2)), ((0, 1), (2, 0)), ((0, 1, 2), (2, 1, 3)), ((0, 1), (0, 1, 2)), ((5, 6), (7, 8)),
                ((0,), (0,)), ((3, 0, 1), (1, 4, 0, 5))]


@pytest.mark.parametrize("kind", ["right", "full"])
@pytest.mark.parametrize("shape", range(len(OUTER_SHAPES)))
@pytest.mark.parametrize("size", [(0, 10), (10, 0), (1, 1), (300, 500), (5000, 40_000)])
def test_outer_joins_random_sets(ctx, orc, kind, shape, size):
    """Right and full outer joins equal the oracle's, unmatched rows padded with 0
    (keys include the unbound value 0, which never matches)."""
    lv, rv = OUTER_SHAPES[shape]
    rng = np.random.default_rng((shape * 7919 + size[0] * 31 + size[1] + (kind == "full")) % 2 ** 32)
    nl, nr = size
    if (lv, rv) == ((5, 6), (7, 8)):  # cross product: keep it small
        nl, nr = min(nl, 300), min(nr, 200)
    hi = max(4, int(np.sqrt(max(nl, nr, 1))) // 2)
    L = orc.TupleSet(lv, orc.canonical(rng.integers(0, hi, (nl, len(lv)))))
    R = orc.TupleSet(rv, orc.canonical(rng.integers(0, hi, (nr, len(rv)))))
    hl = tb.tid_set_from_host(ctx, L.rows, lv)
    hr = tb.tid_set_from_host(ctx, R.rows, rv)
    want = orc.right_join(L, R) if kind == "right" else orc.full_join(L, R)
    _same(_host(tb.tid_join(ctx, hl, hr, kind)), want)
    with pytest.raises(tb.TidError) as e:
        tb.tid_join(ctx, hl, hr, tb.JOIN[kind] | tb.JOIN["hash"])
    assert e.value.code == tb.TID_ERR_ARG
    tb.tid_set_free(hl)
    tb.tid_set_free(hr)


@pytest.mark.parametrize("kind", ["right", "full"])
def test_outer_join_plans(ctx, orc, kind):
    """Star plans on the university store with every join a right or full outer
    join, through tid_exec, against the oracle's evaluation of the same plan."""
    st_np = synth.university_store(1_000_000)
    st = _store(ctx, st_np.s, st_np.p, st_np.o)
    for name, plan in synth.university_plans(st_np)[:8]:
        plan = [dict(nd, algo=kind) if nd["op"] == "join" else nd for nd in plan]
        try:
            _same(_host(tb.tid_exec(ctx, st, plan)), orc.execute(st_np.s, st_np.p, st_np.o, plan))
        except AssertionError as e:
            raise AssertionError(f"{name}: {e}")
    tb.tid_store_free(st)


def test_plan_join_flags_checked_before_running(ctx):
    """A JOIN node with an unknown algorithm or a hash outer join is refused when
    the plan is checked (TID_ERR_ARG), before anything runs."""
    st = synth.tiny_store(10_000)
    store = tb.tid_load(ctx, _dev(st.s), _dev(st.p), _dev(st.o), copy=1)
    p0 = int(st.p[0])
    base = [{"op": "match", "pattern": synth.Pattern(0, p0, 0, var=(0, -1, 1))},
            {"op": "match", "pattern": synth.Pattern(0, p0, 0, var=(1, -1, 2))}]
    for algo in (0x400, 3, tb.TID_JOIN_RIGHT | tb.JOIN["hash"], tb.TID_JOIN_LEFT | tb.JOIN["hash"]):
        plan = base + [{"op": "join", "inputs": [0, 1], "algo": algo}]
        with pytest.raises(tb.TidError) as e:
            tb.tid_exec(ctx, store, plan)
        assert e.value.code == tb.TID_ERR_ARG, algo
    tb.tid_store_free(store)


def test_university_plans_full_size_sampled(ctx, orc):
    """The plans (star, chain, union, filter) on the full 200M-triple store with
    the default join choice, as the benchmark runs them: every sixth plan is
    compared in full with the oracle's evaluation."""
    st_np = synth.university_store(synth.UNI_FULL)
    st = _store(ctx, st_np.s, st_np.p, st_np.o)
    try:
        for name, plan in synth.university_plans(st_np)[::6]:
            try:
                _same(_host(tb.tid_exec(ctx, st, plan)), orc.execute(st_np.s, st_np.p, st_np.o, plan))
            except AssertionError as e:
                raise AssertionError(f"{name}: {e}")
    finally:
        tb.tid_store_free(st)


def test_entailment_full_size_rules_5_and_11(ctx, orc):
    """Rules R5 and R11 (the chains of the schema) on the full 200M-triple store
    plus its RDFS schema, as the benchmark runs them, against the oracle: the
    conclusions and the paper's step counts."""
    st_np = synth.with_schema(synth.university_store(synth.UNI_FULL))
    vocab = synth.rdfs_vocab(st_np.meta["subjects"])
    st = _store(ctx, st_np.s, st_np.p, st_np.o)
    try:
        for rule in (5, 11):
            h, stats = tb.tid_entail(ctx, st, rule, vocab)
            got = tb.tid_set_to_host(h).copy()
            tb.tid_set_free(h)
            want, wstats = orc.entail(st_np.s, st_np.p, st_np.o, rule, vocab)
            assert got.shape == want.rows.shape and np.array_equal(got, want.rows), rule
            assert stats == wstats, (rule, stats, wstats)
    finally:
        tb.tid_store_free(st)
