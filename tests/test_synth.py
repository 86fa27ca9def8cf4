"""Synthetic inputs: seeded, exact size, sets, IDs in range, recipe shape."""
import numpy as np
import pytest

from paper_1807_01409_gb300 import synth


def _is_set(st):
    k = (st.s.astype(np.int64) << 33) ^ (st.p.astype(np.int64) << 20) ^ st.o.astype(np.int64)
    t = np.stack([st.s, st.p, st.o], 1)
    return np.unique(t, axis=0).shape[0] == st.n


def test_tiny_store_recipe():
    st = synth.tiny_store()
    assert st.n == 1_000_000 and st.s.dtype == np.int32
    assert _is_set(st)
    assert st.s.min() >= 1 and st.s.max() <= synth.TINY_SUBJECTS
    assert st.p.min() >= 1 and st.p.max() <= synth.TINY_PREDICATES
    assert st.o.min() >= 1 and st.o.max() <= synth.TINY_OBJECTS
    # Zipf(1.2): rank 1 is the most frequent predicate, with a mass near 1/H(64, 1.2)
    h = np.bincount(st.p)
    assert h.argmax() == 1
    w = np.arange(1, 65.0) ** -1.2
    assert abs(h[1] / st.n - 1 / w.sum()) < 0.02
    # same seed -> same store
    st2 = synth.tiny_store()
    assert np.array_equal(st.s, st2.s) and np.array_equal(st.o, st2.o)


def test_tiny_queries_shapes():
    st = synth.tiny_store()
    q = synth.tiny_queries(st)
    assert [p.shape() for p in q] == ["s??"] * 4 + ["?p?"] * 4 + ["?po"] * 4 + ["sp?"] * 4


def test_university_store_recipe():
    n = 400_000
    st = synth.university_store(n)
    assert st.n == n and _is_set(st)
    lay = synth.uni_layout(synth.uni_subjects(n))
    assert st.s.min() >= 1 and st.s.max() <= synth.uni_subjects(n)
    assert set(np.unique(st.p)) <= set(lay["pred_ids"].tolist())
    lit = st.o >= synth.LIT_BASE
    assert abs(lit.mean() - 0.40) < 0.02           # 40% literal-valued objects
    freq = np.array([(st.p == pid).mean() for pid in lay["pred_ids"]])
    assert np.abs(freq - synth.PRED_FREQ).max() < 0.02
    # type objects are class IDs
    tmask = st.p == lay["pred_ids"][0]
    assert (st.o[tmask] >= lay["class_base"]).all() and (st.o[tmask] < lay["pred_base"]).all()


def test_university_queries_selectivity_span():
    st = synth.university_store(400_000)
    qs = synth.university_queries(st)
    assert len(qs) == 64
    real = np.array([r for _, _, r in qs])
    assert real.max() >= 0.05 and real.min() <= 1e-4


def test_rdfs_schema_is_disjoint_from_the_data():
    st = synth.university_store(200_000)
    v = synth.rdfs_vocab(st.meta["subjects"])
    ss, sp, so = synth.rdfs_schema(st.meta["subjects"])
    assert set(np.unique(sp).tolist()) <= {v["domain"], v["range"], v["subprop"], v["subclass"]}
    assert not set(np.unique(st.p).tolist()) & {v["domain"], v["range"], v["subprop"], v["subclass"]}
    assert v["type"] in set(np.unique(st.p).tolist())
    full = synth.with_schema(st)
    assert np.unique(np.stack([full.s, full.p, full.o], 1), axis=0).shape[0] == full.n
    # the subclass tree: 8 x 511 edges inside the top classes and 7 links between them
    assert int((sp == v["subclass"]).sum()) == 8 * 511 + 7


def test_device_recipe_matches_the_host_recipe_on_cpu():
    """university_store_torch (run here on the CPU) draws a set of exactly n triples
    whose predicate frequencies match the host generator's and whose IDs follow its
    layout."""
    torch = pytest.importorskip("torch")
    n = 400_000
    s, p, o = synth.university_store_torch(n, device="cpu")
    assert s.shape[0] == p.shape[0] == o.shape[0] == n
    assert torch.unique(torch.stack([s, p, o], 1), dim=0).shape[0] == n
    lay = synth.uni_layout(synth.uni_subjects(n))
    pid = lay["pred_ids"]
    freq = np.bincount(p.numpy() - int(pid[0]), minlength=len(pid)) / n
    host = synth.university_store(n)  # the same recipe on the host (duplicates removed the same way)
    hfreq = np.bincount(host.p - int(pid[0]), minlength=len(pid)) / n
    assert np.allclose(freq, hfreq, atol=0.002)
    assert int(s.min()) >= 1 and int(s.max()) <= synth.uni_subjects(n)


def test_batch_queries_sizes_and_shapes():
    """Every drawn query's tally size lies within the window of its target whenever
    such a pattern exists, all seven shapes occur, and the sizes are the value
    tallies of the store."""
    torch = pytest.importorskip("torch")
    s, p, o = synth.university_store_torch(300_000, device="cpu")
    qs = synth.batch_queries(s, p, o, m=700, hi=1e5)
    shapes = {q.shape() for q, _, _ in qs}
    assert len(shapes) == 7, shapes
    within = sum(1 for _, t, sz in qs if t / 1.5 <= sz <= t * 1.5)
    assert within >= 0.9 * len(qs)
    S, P, O = (x.numpy() for x in (s, p, o))
    for q, _, sz in qs[:40]:
        m = np.ones(S.shape[0], bool)
        for col, v in ((S, q.s), (P, q.p), (O, q.o)):
            if v:
                m &= col == v
        assert int(m.sum()) == sz, (q.key(), sz)


def test_serving_requests_stream():
    """Poisson arrivals at the stated rate, the classes in their proportions
    (lookups and wide scans are index requests), wide scans and typed star joins
    present, and every plan well formed (bound slots anonymous, joins on a
    shared variable)."""
    torch = pytest.importorskip("torch")
    s, p, o = synth.university_store_torch(300_000, device="cpu")
    kinds, payloads, arr = synth.serving_requests(s, p, o, m=2000, rate=20000.0)
    assert np.all(np.diff(arr) > 0)
    assert abs(2000 / arr[-1] - 20000.0) < 2000.0
    frac_index = kinds.count("index") / len(kinds)
    assert abs(frac_index - synth.SERVE_MIX[0] - synth.SERVE_MIX[3]) < 0.04
    type_pred = int(synth.uni_layout(synth.uni_subjects(300_000))["pred_ids"][0])
    typed = [x for k, x in zip(kinds, payloads) if k == "plan" and x[0]["pattern"].p == type_pred]
    assert len(typed) >= 10
    sizes = []
    for k, x in zip(kinds, payloads):
        if k == "index":
            key = x.key()
            msk = torch.ones(s.shape[0], dtype=torch.bool)
            for col, v in zip((s, p, o), key):
                if v:
                    msk &= col == v
            sizes.append(int(msk.sum()))
    assert max(sizes) > 0.05 * s.shape[0]  # the wide scans reach large selectivities
    for k, x in zip(kinds, payloads):
        if k == "index":
            assert any(x.key())
            continue
        for nd in x:
            if nd["op"] == "match":
                pat = nd["pattern"]
                assert all(v == -1 for v, key in zip(pat.var, pat.key()) if key)
                assert any(v >= 0 for v in pat.var)
        if x[-1]["op"] == "join":
            a, b = (x[i]["pattern"] for i in x[-1]["inputs"])
            assert {v for v in a.var if v >= 0} & {v for v in b.var if v >= 0}
