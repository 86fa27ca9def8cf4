"""Batched single-pattern search (tid_match_batch) through the C ABI against the
CPU oracle, bit-exact: every bound-position mask, ragged sizes, repeated and
absent keys, more distinct keys than one sub-batch holds, and a 4096-query batch
of log-uniform result sizes on a large store (sampled lists against the oracle,
every list against its size from the store's value tallies)."""
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


def _lists(handles):
    out = []
    for h in handles:
        out.append(tb.tid_set_to_host(h)[:, 0].copy())
        tb.tid_set_free(h)
    return out


def _all_keys(ns, np_, no):
    keys = []
    for s in range(ns + 1):
        for p in range(np_ + 1):
            for o in range(no + 1):
                keys.append((s, p, o))
    return keys


@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 256, 257, 4097, 100_003, 1_000_001])
def test_every_mask_ragged(ctx, orc, n):
    rng = np.random.default_rng(n + 11)
    S = rng.integers(1, 4, n).astype(np.int32)
    P = rng.integers(1, 3, n).astype(np.int32)
    O = rng.integers(1, 5, n).astype(np.int32)
    store = tb.tid_load(ctx, _dev(S), _dev(P), _dev(O), copy=1)
    keys = _all_keys(4, 3, 5)  # includes (?,?,?) and absent values
    got = _lists(tb.tid_match_batch(ctx, store, keys))
    for k, g in zip(keys, got):
        assert np.array_equal(g, orc.match(S, P, O, k)), (n, k)
    tb.tid_store_free(store)


def test_tiny_store_with_repeats(ctx, orc):
    st = synth.tiny_store()
    store = tb.tid_load(ctx, *[_dev(c) for c in (st.s, st.p, st.o)], copy=0)
    qs = [q.key() for q in synth.tiny_queries(st)]
    keys = qs + qs[::-1] + [(0, 0, 0), (10 ** 9, 0, 0)]
    got = _lists(tb.tid_match_batch(ctx, store, keys))
    for k, g in zip(keys, got):
        assert np.array_equal(g, orc.match(st.s, st.p, st.o, k)), k
    tb.tid_store_free(store)


def test_more_keys_than_one_sub_batch(ctx, orc):
    """More than twice TID_BATCH_KEYS distinct keys of all seven masks: three sub-batches."""
    st = synth.tiny_store()
    store = tb.tid_load(ctx, *[_dev(c) for c in (st.s, st.p, st.o)], copy=0)
    rng = np.random.default_rng(5)
    rows = rng.integers(0, st.n, 3 * tb.TID_BATCH_KEYS)
    keys = []
    for i, r in enumerate(rows):
        m = 1 + i % 7
        t = (int(st.s[r]), int(st.p[r]), int(st.o[r]))
        keys.append(tuple(t[j] if (m >> j) & 1 else 0 for j in range(3)))
    got = _lists(tb.tid_match_batch(ctx, store, keys))
    assert len(set(keys)) > 2 * tb.TID_BATCH_KEYS
    for k, g in zip(keys, got):
        assert np.array_equal(g, orc.match(st.s, st.p, st.o, k)), k
    tb.tid_store_free(store)


def test_empty_batch_and_empty_store(ctx, orc):
    store = tb.tid_load(ctx, np.ones(5, np.int32), np.ones(5, np.int32), np.ones(5, np.int32))
    assert tb.tid_match_batch(ctx, store, []) == []
    tb.tid_store_free(store)
    empty = tb.tid_load(ctx, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    got = _lists(tb.tid_match_batch(ctx, empty, [(1, 0, 0), (0, 0, 0)]))
    assert all(g.shape[0] == 0 for g in got)
    tb.tid_store_free(empty)


def test_negative_id_rejected(ctx):
    store = tb.tid_load(ctx, np.ones(4, np.int32), np.ones(4, np.int32), np.ones(4, np.int32))
    with pytest.raises(tb.TidError) as e:
        tb.tid_match_batch(ctx, store, [(1, 0, 0), (0, -3, 0)])
    assert e.value.code == tb.TID_ERR_ID
    tb.tid_store_free(store)


def test_equals_single_launches_on_university(ctx, orc):
    """A 64-query batch on the 20M university store equals the oracle list by list."""
    st = synth.university_store(20_000_000)
    store = tb.tid_load(ctx, *[_dev(c) for c in (st.s, st.p, st.o)], copy=0)
    keys = [pat.key() for pat, _, _ in synth.university_queries(st)]
    got = _lists(tb.tid_match_batch(ctx, store, keys))
    for k, g in zip(keys, got):
        assert np.array_equal(g, orc.match(st.s, st.p, st.o, k)), k
    tb.tid_store_free(store)


def test_large_store_4096_queries(ctx, orc):
    """The batched workload: 500M triples, 4096 queries with log-uniform result sizes
    in [1, 1e7].  Every list is ascending, answers its pattern and has the size the
    store's value tallies give; 24 lists are compared in full with the oracle."""
    n = 500_000_000
    s, p, o = synth.university_store_torch(n, device="cuda")
    qs = synth.batch_queries(s, p, o)
    keys = [pat.key() for pat, _, _ in qs]
    store = tb.tid_load(ctx, s, p, o, copy=0)
    handles = tb.tid_match_batch(ctx, store, keys)
    hs, hp, ho = (t.cpu().numpy() for t in (s, p, o))
    sample = set(np.random.default_rng(3).choice(len(keys), 24, replace=False).tolist())
    for i, ((pat, _, size), h) in enumerate(zip(qs, handles)):
        g = tb.tid_set_to_host(h)[:, 0]
        tb.tid_set_free(h)
        assert g.shape[0] == size, (pat.key(), g.shape[0], size)
        if g.shape[0]:
            assert np.all(np.diff(g) > 0)
            for col, v in ((hs, pat.s), (hp, pat.p), (ho, pat.o)):
                if v:
                    assert np.all(col[g] == v), pat.key()
        if i in sample:
            assert np.array_equal(g, orc.match(hs, hp, ho, pat.key())), pat.key()
    tb.tid_store_free(store)
