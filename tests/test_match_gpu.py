"""K1 (single-pattern scan + compaction) through the C ABI against the CPU
oracle, bit-exact: the paper's worked example, the 1M Zipf store, ragged and
degenerate sizes, every bound-column mask, misaligned borrowed columns, and
the full 200M university store in the configuration the benchmark times."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def _match(ctx, store, key):
    h = tb.tid_match(ctx, store, key)
    try:
        return tb.tid_set_to_host(h)[:, 0].copy()
    finally:
        tb.tid_set_free(h)


def test_worked_example_rule11(ctx, orc):
    g = json.load(open(os.path.join(GOLDEN, "rule11_worked_example.json")))
    st = np.array(g["store"], np.int32)
    store = tb.tid_load(ctx, st[:, 0].copy(), st[:, 1].copy(), st[:, 2].copy())
    idx = _match(ctx, store, tuple(g["step1"]["key"]))
    flags = np.zeros(len(st), int)
    flags[idx] = 1
    assert flags.tolist() == g["step1"]["flags"]
    flags2 = np.zeros(len(st), int)
    for k in g["step2"]["keys"]:
        flags2[_match(ctx, store, tuple(k))] = 1
    assert flags2.tolist() == g["step2"]["flags"]
    tb.tid_store_free(store)


def test_tiny_store_queries(ctx, orc):
    st = synth.tiny_store()
    cols = [_dev(c) for c in (st.s, st.p, st.o)]
    store = tb.tid_load(ctx, *cols, copy=0)
    for q in synth.tiny_queries(st) + [synth.Pattern(0, 0, 0)]:
        got = _match(ctx, store, q)
        want = orc.match(st.s, st.p, st.o, q.key())
        assert np.array_equal(got, want), q.key()
    tb.tid_store_free(store)


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 1023, 4095, 4096, 4097, 8191, 12289, 100_003, 1_000_001])
def test_ragged_sizes_all_masks(ctx, orc, n):
    rng = np.random.default_rng(n)
    S = rng.integers(1, 4, n).astype(np.int32)
    P = rng.integers(1, 3, n).astype(np.int32)
    O = rng.integers(1, 5, n).astype(np.int32)
    store = tb.tid_load(ctx, _dev(S), _dev(P), _dev(O), copy=1)
    for key in [(0, 0, 0), (2, 0, 0), (0, 1, 0), (0, 0, 3), (1, 2, 0), (3, 0, 4), (0, 2, 2), (1, 1, 1),
                (9, 0, 0)]:
        assert np.array_equal(_match(ctx, store, key), orc.match(S, P, O, key)), (n, key)
    tb.tid_store_free(store)


@pytest.mark.parametrize("off", [1, 2, 3])
def test_misaligned_borrowed_columns(ctx, orc, off):
    """Columns that start off a 16-byte boundary take the scalar-load path."""
    n = 50_000 + off
    rng = np.random.default_rng(off)
    base = [torch.from_numpy(rng.integers(1, 6, n + 8).astype(np.int32)).cuda() for _ in range(3)]
    cols = [b[off:off + n] for b in base]
    store = tb.tid_load(ctx, *cols, copy=0)
    host = [c.cpu().numpy() for c in cols]
    for key in [(3, 0, 0), (0, 2, 5), (1, 1, 1), (0, 0, 0)]:
        assert np.array_equal(_match(ctx, store, key), orc.match(*host, key))
    tb.tid_store_free(store)


def test_dense_and_empty_results(ctx, orc):
    n = 300_000
    S = np.arange(1, n + 1, dtype=np.int32)
    P = np.ones(n, np.int32)
    O = np.full(n, 7, np.int32)
    store = tb.tid_load(ctx, S, P, O)  # from host memory
    assert np.array_equal(_match(ctx, store, (0, 1, 0)), np.arange(n, dtype=np.int32))
    assert np.array_equal(_match(ctx, store, (0, 1, 7)), np.arange(n, dtype=np.int32))
    assert _match(ctx, store, (0, 2, 0)).shape[0] == 0
    assert np.array_equal(_match(ctx, store, (n, 1, 7)), np.array([n - 1], np.int32))
    tb.tid_store_free(store)


def test_negative_id_rejected(ctx):
    store = tb.tid_load(ctx, np.ones(4, np.int32), np.ones(4, np.int32), np.ones(4, np.int32))
    with pytest.raises(tb.TidError) as e:
        tb.tid_match(ctx, store, (0, -3, 0))
    assert e.value.code == tb.TID_ERR_ID
    tb.tid_store_free(store)


def test_back_to_back_launches_without_sync(ctx, orc):
    """Many matches queued before any wait: ticket and epoch reuse across launches."""
    st = synth.tiny_store()
    store = tb.tid_load(ctx, *[_dev(c) for c in (st.s, st.p, st.o)], copy=0)
    qs = synth.tiny_queries(st) * 4
    handles = [tb.tid_match(ctx, store, q) for q in qs]
    for q, h in zip(qs, handles):
        got = tb.tid_set_to_host(h)[:, 0]
        assert np.array_equal(got, orc.match(st.s, st.p, st.o, q.key()))
        tb.tid_set_free(h)
    tb.tid_store_free(store)


def test_university_full_size_all_queries(ctx, orc):
    """The benchmark's workload: 200M triples, 64 queries, every index list
    compared in full with the oracle."""
    st = synth.university_store()
    qs = synth.university_queries(st)
    store = tb.tid_load(ctx, *[_dev(c) for c in (st.s, st.p, st.o)], copy=0)
    for pat, _, _ in qs:
        got = _match(ctx, store, pat)
        want = orc.match(st.s, st.p, st.o, pat.key())
        assert np.array_equal(got, want), pat.key()
    tb.tid_store_free(store)


def test_concurrent_contexts(ctx, orc):
    """Two host threads, each with its own context and stream, scan at the same time
    (the scan is a cooperative launch whose grid fills the GPU): every result equals
    the oracle's and no in-kernel wait gives up."""
    import threading
    st = synth.university_store(20_000_000)
    qs = [q for q, _, _ in synth.university_queries(st)][:24]
    cols = [_dev(c) for c in (st.s, st.p, st.o)]
    torch.cuda.synchronize()
    want = {q.key(): orc.match(st.s, st.p, st.o, q.key()) for q in qs}
    errors = []

    def worker(order):
        c = tb.tid_ctx_create(0, None)
        try:
            store = tb.tid_load(c, *cols, copy=0)
            for _ in range(3):
                hs = [(q, tb.tid_match(c, store, q)) for q in order]
                for q, h in hs:
                    got = tb.tid_set_to_host(h)[:, 0]
                    tb.tid_set_free(h)
                    if not np.array_equal(got, want[q.key()]):
                        errors.append(q.key())
            tb.tid_store_free(store)
        except Exception as e:  # reported below
            errors.append(repr(e))
        finally:
            tb.tid_ctx_destroy(c)

    ths = [threading.Thread(target=worker, args=(qs,)), threading.Thread(target=worker, args=(qs[::-1],))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errors, errors[:5]
