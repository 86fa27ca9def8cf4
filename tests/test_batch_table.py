"""The key tables of the batched search (tid_match_batch), checked on the CPU
through the C ABI: tid_batch_table_check runs the batch's host-side planning
(distinct keys, sub-batches, one perfect-hash table per sub-batch) and then
looks every key up the way the kernel does.  A batch of distinct keys must
always be planned -- keys whose IDs have arithmetic structure (powers of two
apart, entity and literal IDs 2^30 apart, the largest IDs) included -- on
every seed."""
import itertools

import numpy as np
import pytest

from paper_1807_01409_gb300 import binding as tb


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1807_01409_gb300 import build
    build.build()


def _all_keys(vals):
    """Every (s, p, o) over vals and the wildcard 0, except (?, ?, ?)."""
    vals = [0] + [int(v) for v in vals]
    return [k for k in itertools.product(vals, vals, vals) if k != (0, 0, 0)]


EXTREME = [1, 2, 2 ** 30 - 1, 2 ** 30, 2 ** 31 - 2, 2 ** 31 - 1]


def test_extreme_ids_on_a_thousand_seeds():
    """The 342 keys over IDs at both ends of the positive int32 range (the set a
    linear hash cannot separate) get a table on every one of 1000 seeds, almost
    always at the first seed tried."""
    keys = _all_keys(EXTREME)
    assert len(keys) == 342
    first_try = 0
    for seed in range(1000):
        rc, tries, subs = tb.tid_batch_table_check(keys, seed * 0x9E3779B9)
        assert rc == tb.TID_OK, (seed, tb.last_error())
        assert subs >= 1
        first_try += tries == 1
    assert first_try >= 990, first_try


def test_entity_and_literal_ids_2_30_apart():
    """Entity IDs e and literal IDs e + 2^30 in every column, with compensating
    differences in the other columns: every seed plans the batch."""
    rng = np.random.default_rng(5)
    for seed in range(1000):
        e = rng.integers(1, 2 ** 30 - 4, 4)
        vals = sorted(set(int(v) for v in np.r_[e, e + 2 ** 30, e + 1, e + 1 + 2 ** 30]))
        keys = [k for k in _all_keys(vals[:6])]
        rc, tries, subs = tb.tid_batch_table_check(keys, seed)
        assert rc == tb.TID_OK, (seed, tb.last_error())


def test_large_batches_split_into_sub_batches():
    """Batches above one sub-batch (TID_BATCH_KEYS distinct keys) are split, and
    duplicate patterns share a key."""
    rng = np.random.default_rng(11)
    n = 5000
    masks = rng.integers(1, 8, n)
    vals = rng.integers(1, 2 ** 31 - 1, (n, 3))
    keys = [tuple(int(vals[i, c]) if (masks[i] >> c) & 1 else 0 for c in range(3)) for i in range(n)]
    keys = keys + keys[:700]  # repeats
    for seed in (0, 1, 2 ** 32 - 1):
        rc, tries, subs = tb.tid_batch_table_check(keys, seed)
        assert rc == tb.TID_OK, tb.last_error()
        assert subs == -(-n // tb.TID_BATCH_KEYS), subs


def test_degenerate_batches():
    assert tb.tid_batch_table_check([], 0)[0] == tb.TID_OK
    assert tb.tid_batch_table_check([(0, 0, 0)], 0)[:3] == (tb.TID_OK, 0, 0)
    assert tb.tid_batch_table_check([(5, 0, 0)], 0)[0] == tb.TID_OK
    assert tb.tid_batch_table_check([(5, -1, 0)], 0)[0] == tb.TID_ERR_ID
