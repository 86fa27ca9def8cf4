"""Failure handling without a GPU fault: device allocations are refused on the
host (tid_ctx_inject_alloc_failure) at every point of each operator in turn.
Every call either succeeds with the oracle's result or fails with TID_ERR_OOM
and no output; afterwards the same context answers correctly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1807_01409_gb300 import binding as tb
from paper_1807_01409_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    from paper_1807_01409_gb300 import build
    build.build()
    st = synth.with_schema(synth.university_store(300_000))
    ctx = tb.tid_ctx_create(0, None)
    store = tb.tid_load(ctx, st.s, st.p, st.o)
    yield ctx, store, st
    tb.tid_store_free(store)
    tb.tid_ctx_destroy(ctx)


def _rows(h):
    try:
        return tb.tid_set_to_host(h).copy()
    finally:
        tb.tid_set_free(h)


def _ops(ctx, store, st, orc):
    """(name, call returning host rows, expected rows) for each operator."""
    q = [p for p, _, _ in synth.university_queries(st)]
    key = q[3].key()
    plans = synth.university_plans(st)
    star = next(pl for name, pl in plans if name.startswith("star"))
    vocab = synth.rdfs_vocab(st.meta["subjects"])
    X, Y = 0, 1
    pat_a = synth.Pattern(0, int(st.p[0]), 0, var=(X, -1, Y))
    idx_a = orc.match(st.s, st.p, st.o, pat_a.key())
    bound = orc.bind(st.s, st.p, st.o, pat_a.key(), pat_a.var, idx_a)

    def match():
        return _rows(tb.tid_match(ctx, store, key))

    def batch():
        hs = tb.tid_match_batch(ctx, store, [x.key() for x in q[:12]])
        return np.concatenate([_rows(h)[:, 0] for h in hs])

    def multi():
        hs = tb.tid_match_multi(ctx, store, q[:3])
        return np.concatenate([_rows(h)[:, 0] for h in hs])

    def bind():
        i = tb.tid_match(ctx, store, pat_a)
        try:
            return _rows(tb.tid_bind(ctx, store, pat_a, i))
        finally:
            tb.tid_set_free(i)

    def execute():
        return _rows(tb.tid_exec(ctx, store, star))

    def entail():
        h, _ = tb.tid_entail(ctx, store, 9, vocab)
        return _rows(h)

    want_batch = np.concatenate([orc.match(st.s, st.p, st.o, x.key()) for x in q[:12]])
    want_multi = np.concatenate([orc.match(st.s, st.p, st.o, x.key()) for x in q[:3]])
    return [
        ("match", match, orc.match(st.s, st.p, st.o, key).reshape(-1, 1)),
        ("batch", batch, want_batch),
        ("multi", multi, want_multi),
        ("bind", bind, bound.rows),
        ("exec", execute, orc.execute(st.s, st.p, st.o, star).rows),
        ("entail", entail, orc.entail(st.s, st.p, st.o, 9, vocab)[0].rows),
    ]


def test_every_operator_fails_cleanly_and_recovers(env, orc):
    ctx, store, st = env
    for name, call, want in _ops(ctx, store, st, orc):
        failures = 0
        for after in range(0, 64):
            tb.tid_ctx_inject_alloc_failure(ctx, after)
            try:
                got = call()
                ok = True
            except tb.TidError as e:
                assert e.code == tb.TID_ERR_OOM, (name, after, e)
                ok = False
            finally:
                tb.tid_ctx_inject_alloc_failure(ctx, -1)
            if ok:  # enough allocations for the whole call
                assert np.array_equal(got, want), (name, after)
                break
            failures += 1
            # the context still answers after a refused allocation
            assert np.array_equal(call(), want), (name, after)
        assert failures > 0, name  # the call allocates, so the first points must fail
    tb.tid_ctx_sync(ctx)
