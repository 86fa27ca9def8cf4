"""The request server (tid_server_*) through the C ABI: every result equals the
CPU oracle's, a request's result is the same alone and in a mixed stream (bit
for bit), the batched and the one-request-at-a-time configurations agree,
admission respects the budget, and bad requests fail at submission."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1807_01409_gb300 import binding as tb
from paper_1807_01409_gb300 import synth

pytestmark = pytest.mark.gpu

N = 2_000_000


@pytest.fixture(scope="module")
def store():
    from paper_1807_01409_gb300 import build
    build.build()
    st = synth.university_store(N)
    cols = tuple(torch.from_numpy(c).cuda() for c in (st.s, st.p, st.o))
    torch.cuda.synchronize()
    return st, cols


@pytest.fixture(scope="module")
def requests(store):
    _, (s, p, o) = store
    kinds, payloads, _ = synth.serving_requests(s, p, o, m=300, seed=11)
    return list(zip(kinds, payloads))


def _submit(srv, kind, x):
    return srv.submit_index(x) if kind == "index" else srv.submit_plan(x)


def _want(orc, st, kind, x):
    if kind == "index":
        return (-1,), orc.match(st.s, st.p, st.o, x.key()).reshape(-1, 1)
    t = orc.execute(st.s, st.p, st.o, x)
    return tuple(t.vars), t.rows


def _run_all(srv, reqs):
    ids = [_submit(srv, k, x) for k, x in reqs]
    out = []
    for i in ids:
        assert srv.wait(i, 60_000)
        status, vars_, rows, lat = srv.result(i)
        assert status == tb.TID_OK
        assert lat > 0
        out.append((vars_, rows))
    return out


def test_mixed_stream_equals_oracle(store, requests, orc):
    st, cols = store
    with tb.Server(*cols, workers=2, max_wave=64) as srv:
        got = _run_all(srv, requests)
        stats = srv.stats()
    assert stats["completed"] == len(requests) and stats["failed"] == 0
    assert stats["max_wave_seen"] > 1
    for (kind, x), (gv, gr) in zip(requests, got):
        wv, wr = _want(orc, st, kind, x)
        assert gv == wv, (kind, gv, wv)
        assert gr.shape == wr.shape and np.array_equal(gr, wr), kind


def test_alone_equals_in_the_mix(store, requests):
    """Each request submitted alone to an idle server returns exactly what it
    returned inside the mixed stream (tolerance 0: integer results)."""
    _, cols = store
    with tb.Server(*cols, workers=2, max_wave=4096) as srv:
        mixed = _run_all(srv, requests)
        for (kind, x), (mv, mr) in zip(requests[::7], mixed[::7]):
            (av, ar), = _run_all(srv, [(kind, x)])
            assert av == mv and np.array_equal(ar, mr), kind


def test_plain_configuration_agrees(store, requests):
    """One request at a time, each searching alone (one launch per query), gives the
    same results as the batched configuration."""
    _, cols = store
    with tb.Server(*cols, workers=1, max_wave=1, batch_scans=False) as plain:
        a = _run_all(plain, requests[:120])
        sp = plain.stats()
    with tb.Server(*cols, workers=3, max_wave=32, batch_scans=True) as batched:
        b = _run_all(batched, requests[:120])
    assert sp["max_wave_seen"] == 1
    for (av, ar), (bv, br) in zip(a, b):
        assert av == bv and np.array_equal(ar, br)


def test_budget_admits_one_at_a_time(store, requests):
    """A budget below every estimate admits each request alone (the head of the
    queue always runs when nothing else is admitted)."""
    _, cols = store
    with tb.Server(*cols, workers=2, max_wave=64, budget_bytes=1) as srv:
        _run_all(srv, requests[:40])
        st = srv.stats()
    assert st["max_wave_seen"] == 1
    assert st["completed"] == 40


def test_submission_errors(store):
    _, cols = store
    with tb.Server(*cols, workers=1, max_wave=8) as srv:
        with pytest.raises(tb.TidError) as e:
            srv.submit_index((0, -1, 0))
        assert e.value.code == tb.TID_ERR_ID
        with pytest.raises(tb.TidError):
            srv.submit_plan([{"op": "join", "inputs": [0, 1]}])
        with pytest.raises(tb.TidError):
            srv.wait(10 ** 9)
        rid = srv.submit_index((0, int(cols[1][0]), 0))
        assert srv.wait(rid)
        srv.release(rid)
        with pytest.raises(tb.TidError):
            srv.result(rid)


def test_concurrent_submitters(store, requests, orc):
    """Requests submitted from several host threads at once."""
    import threading
    st, cols = store
    chunks = [requests[i::4] for i in range(4)]
    results = [None] * 4
    with tb.Server(*cols, workers=2, max_wave=128) as srv:
        def go(j):
            results[j] = _run_all(srv, chunks[j])
        ths = [threading.Thread(target=go, args=(j,)) for j in range(4)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    for j in range(4):
        for (kind, x), (gv, gr) in list(zip(chunks[j], results[j]))[::5]:
            wv, wr = _want(orc, st, kind, x)
            assert gv == wv and np.array_equal(gr, wr)


def test_large_index_results_in_chunks(orc):
    """Index results longer than one pinned staging buffer (16M rows) reach the
    host in several chunks, in a wave with small requests, each equal to the
    oracle's list."""
    rng = np.random.default_rng(77)
    n = 40_000_003
    S = rng.integers(1, 50_000, n, dtype=np.int32)
    P = rng.integers(1, 3, n, dtype=np.int32)  # two predicates: (?, 1, ?) holds ~20M rows
    O = rng.integers(1, 1000, n, dtype=np.int32)
    cols = tuple(torch.from_numpy(c).cuda() for c in (S, P, O))
    torch.cuda.synchronize()
    keys = [(0, 1, 0), (int(S[5]), 0, 0), (0, 2, int(O[7])), (0, 2, 0), (int(S[9]), int(P[9]), 0)]
    with tb.Server(*cols, workers=1, max_wave=64) as srv:
        got = _run_all(srv, [("index", k) for k in keys])
    for k, (gv, gr) in zip(keys, got):
        want = orc.match(S, P, O, k)
        assert gv == (-1,) and gr.shape == (want.shape[0], 1), k
        assert np.array_equal(gr[:, 0], want), k
    assert max(g[1].shape[0] for g in got) > 16_000_000
