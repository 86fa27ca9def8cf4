"""The operators at the sizes of the multi-pattern workload (intermediate
results of tens of millions of tuples, Section 4.2 and 4.3), through the C ABI
against the CPU oracle's sort-merge path, element by element: the canonical
sort (packed keys and the row permutation), joins of 8M-row inputs with both
algorithms, union and projection of 30M rows.  Collected after the other
operator files."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1807_01409_gb300 import binding as tb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1807_01409_gb300 import build
    build.build()
    c = tb.tid_ctx_create(0, None)
    yield c
    tb.tid_ctx_destroy(c)


def _host(h):
    try:
        return tuple(tb.tid_set_info(h)["vars"]), tb.tid_set_to_host(h).copy()
    finally:
        tb.tid_set_free(h)


def _same(got, want):
    gv, gr = got
    assert gv == tuple(want.vars), (gv, want.vars)
    assert gr.shape == want.rows.shape, (gr.shape, want.rows.shape)
    assert np.array_equal(gr, want.rows)


def _rows(rng, n, highs):
    return np.stack([rng.integers(1, h, n, dtype=np.int64) for h in highs], axis=1).astype(np.int32)


@pytest.mark.parametrize("highs", [(5_000_000, 2 ** 30 + 10_000_000),           # packed 64-bit keys
                                   (2 ** 31 - 1, 2 ** 31 - 1, 2 ** 31 - 1),       # row permutation
                                   (5_000_000, 20, 2 ** 30 + 2 ** 20, 4096)])   # four columns
def test_canonical_sort_20M(ctx, orc, highs):
    """Sets of 20M rows in 2-4 columns put into canonical order (with
    duplicates) equal the oracle's canonical form."""
    rng = np.random.default_rng(len(highs) * 101 + highs[0] % 97)
    rows = _rows(rng, 20_000_000, highs)
    rows[rng.integers(0, rows.shape[0], 100_000)] = rows[0]  # duplicates
    vars_ = tuple(range(len(highs)))
    got = _host(tb.tid_set_from_host(ctx, rows, vars_))
    _same(got, orc.TupleSet(vars_, orc.canonical(rows)))


@pytest.mark.parametrize("algo", ["sort_merge", "hash"])
@pytest.mark.parametrize("shape", ["prefix", "second_column", "star_bench"])
def test_join_8M(ctx, orc, algo, shape):
    """Joins of canonical inputs of millions of rows: on the leading column of
    both (a subject star), on a column that leads neither, and the bench's
    0.5M x 8.2M shape."""
    rng = np.random.default_rng({"prefix": 1, "second_column": 2, "star_bench": 3}[shape])
    if shape == "star_bench":
        L = orc.TupleSet((0, 1), orc.canonical(_rows(rng, 500_000, (5_000_000, 2 ** 30 + 10 ** 6))))
        R = orc.TupleSet((0, 2), orc.canonical(_rows(rng, 8_200_000, (5_000_000, 5_000_512))))
    elif shape == "prefix":
        L = orc.TupleSet((0, 1), orc.canonical(_rows(rng, 8_000_000, (4_000_000, 1_000_000))))
        R = orc.TupleSet((0, 2), orc.canonical(_rows(rng, 8_000_000, (4_000_000, 2 ** 30 + 10 ** 7))))
    else:
        L = orc.TupleSet((1, 0), orc.canonical(_rows(rng, 8_000_000, (1_000_000, 4_000_000))))
        R = orc.TupleSet((2, 0, 3), orc.canonical(_rows(rng, 8_000_000, (2 ** 30 + 10 ** 7, 4_000_000, 64))))
    hl = tb.tid_set_from_host(ctx, L.rows, L.vars)
    hr = tb.tid_set_from_host(ctx, R.rows, R.vars)
    try:
        want = orc.join(L, R, "sortmerge")
        assert want.n > 500_000
        _same(_host(tb.tid_join(ctx, hl, hr, algo)), want)
    finally:
        tb.tid_set_free(hl)
        tb.tid_set_free(hr)


def test_union_and_project_30M(ctx, orc):
    """Union of two overlapping 16M-row sets, one lacking a variable (padded
    with 0), and the projection of the 30M-row result on two of its variables,
    equal the oracle's."""
    rng = np.random.default_rng(30)
    a = _rows(rng, 16_000_000, (5_000_000, 30, 2 ** 30 + 10 ** 6))
    b = np.concatenate([a[rng.integers(0, a.shape[0], 2_000_000)][:, [0, 2]],
                        _rows(rng, 14_000_000, (5_000_000, 2 ** 30 + 10 ** 6))])
    A = orc.TupleSet((0, 1, 2), orc.canonical(a))
    B = orc.TupleSet((0, 2), orc.canonical(b))
    ha = tb.tid_set_from_host(ctx, A.rows, A.vars)
    hb = tb.tid_set_from_host(ctx, B.rows, B.vars)
    try:
        want = orc.union([A, B])
        assert want.n > 28_000_000
        hu = tb.tid_union(ctx, [ha, hb])
        try:
            _same(_host(tb.tid_project(ctx, hu, [2, 0])), orc.project(want, (2, 0)))
            _same((tuple(tb.tid_set_info(hu)["vars"]), tb.tid_set_to_host(hu)), want)
        finally:
            tb.tid_set_free(hu)
    finally:
        tb.tid_set_free(ha)
        tb.tid_set_free(hb)
