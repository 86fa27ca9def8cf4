"""Synthetic inputs: seeded, exact size, sets, IDs in range, recipe shape."""
import numpy as np

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
