"""RDFS entailment (tid_entail) through the C ABI against the CPU oracle,
bit-exact: the paper's Rule-11 walk-through, all six rules on a university
store with its schema (conclusions and the paper's step counts), the same
store with its IDs spread over the int32 range (so two-term conclusions join
and sort instead of using the pair bit matrix), rules whose schema premise
finds nothing, and bad arguments."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _host(h):
    try:
        return tb.tid_set_to_host(h)
    finally:
        tb.tid_set_free(h)


def test_rule11_worked_example(ctx):
    g = json.load(open(os.path.join(GOLDEN, "rule11_worked_example.json")))
    a = np.array(g["store"], np.int32)
    st = tb.tid_load(ctx, a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy())
    vocab = {"type": 1, "domain": 2, "range": 3, "subprop": 4, "subclass": 84}
    h, stats = tb.tid_entail(ctx, st, 11, vocab)
    rows = _host(h)
    assert sorted(map(tuple, rows.tolist())) == sorted((x, 84, z) for x, z in g["result_xz"])
    assert stats == {"res1": 4, "dist1": 3, "res2": 2, "dist2": 1, "all": 2}
    tb.tid_store_free(st)


@pytest.mark.parametrize("n", [300_000, 2_000_000])
def test_all_rules_equal_oracle(ctx, orc, n):
    st_np = synth.with_schema(synth.university_store(n))
    vocab = synth.rdfs_vocab(st_np.meta["subjects"])
    cols = [torch.from_numpy(c).cuda() for c in (st_np.s, st_np.p, st_np.o)]
    st = tb.tid_load(ctx, *cols, copy=0)
    for rule in tb.RULES:
        h, stats = tb.tid_entail(ctx, st, rule, vocab)
        got = _host(h)
        want, wstats = orc.entail(st_np.s, st_np.p, st_np.o, rule, vocab)
        assert got.shape == want.rows.shape and np.array_equal(got, want.rows), rule
        assert stats == wstats, (rule, stats, wstats)
    tb.tid_store_free(st)


def test_all_rules_sparse_ids_equal_oracle(ctx, orc):
    """The same store with its IDs spread over the int32 range (order kept).  A
    two-term conclusion's pair matrix is then far too large, so every rule
    joins and sorts instead; the results are the oracle's all the same."""
    base = synth.with_schema(synth.university_store(300_000))
    vocab = synth.rdfs_vocab(base.meta["subjects"])
    u = np.unique(np.concatenate([base.s, base.p, base.o]))
    rng = np.random.default_rng(7)
    gap = (2**31 - 2) // u.shape[0]
    new = np.cumsum(rng.integers(1, gap + 1, size=u.shape[0])).astype(np.int64)
    assert new[-1] < 2**31 - 1 and new[-1] - new[0] > 2**30
    s, p, o = (new[np.searchsorted(u, c)].astype(np.int32) for c in (base.s, base.p, base.o))
    assert all(np.isin(v, u) for v in vocab.values())
    vocab = {k: int(new[np.searchsorted(u, v)]) for k, v in vocab.items()}
    st = tb.tid_load(ctx, s, p, o)
    for rule in tb.RULES:
        h, stats = tb.tid_entail(ctx, st, rule, vocab)
        got = _host(h)
        want, wstats = orc.entail(s, p, o, rule, vocab)
        assert got.shape == want.rows.shape and np.array_equal(got, want.rows), rule
        assert stats == wstats, (rule, stats, wstats)
    tb.tid_store_free(st)


def test_schema_premise_absent(ctx, orc):
    """Without schema triples every rule concludes nothing."""
    st_np = synth.university_store(300_000)
    vocab = synth.rdfs_vocab(st_np.meta["subjects"])
    st = tb.tid_load(ctx, st_np.s, st_np.p, st_np.o)
    for rule in tb.RULES:
        h, stats = tb.tid_entail(ctx, st, rule, vocab)
        assert _host(h).shape == (0, 3)
        assert stats["res1"] == 0 and stats["all"] == 0
    tb.tid_store_free(st)


def test_bad_arguments(ctx):
    st = tb.tid_load(ctx, np.ones(4, np.int32), np.ones(4, np.int32), np.ones(4, np.int32))
    vocab = {"type": 1, "domain": 2, "range": 3, "subprop": 4, "subclass": 5}
    with pytest.raises(tb.TidError) as e:
        tb.tid_entail(ctx, st, 4, vocab)
    assert e.value.code == tb.TID_ERR_ARG
    with pytest.raises(tb.TidError) as e:
        tb.tid_entail(ctx, st, 11, dict(vocab, subclass=0))
    assert e.value.code == tb.TID_ERR_ID
    tb.tid_store_free(st)
