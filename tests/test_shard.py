"""Store shards (Section 3's per-GPU chunks) on the CPU: the ranges partition
the store in rank order with aligned inner boundaries, and gathering every
shard's list (gloo ranks) gives the whole store's list.  Each rank's local list
comes from the oracle run on its shard, standing in for the device search."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1807_01409_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("n", [0, 1, 3, 7, 8, 1000, 1001, 123457])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_ranges_partition_the_store(n, world):
    prev_end = 0
    for r in range(world):
        base, m = shard.shard_range(n, world, r)
        assert base == prev_end and m >= 0
        if r < world - 1:
            assert (base + m) % shard.ALIGN == 0
        prev_end = base + m
    assert prev_end == n
    sizes = [shard.shard_range(n, world, r)[1] for r in range(world)]
    assert max(sizes) - min(sizes) <= 2 * shard.ALIGN  # near-equal


def test_bad_arguments():
    for args in ((10, 0, 0), (10, 2, 2), (10, 2, -1), (-1, 2, 0)):
        with pytest.raises(ValueError):
            shard.shard_range(*args)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    from paper_1807_01409_gb300 import shard as sh
    from paper_1807_01409_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st = synth.university_store(40_001)
        keys = [x.key() for x, _, _ in synth.university_queries(st)[:10]] + [(0, 0, 0)]
        base, m = sh.shard_range(st.n, world, rank)
        ok = []
        for key in keys:
            local = orc.match(st.s[base:base + m], st.p[base:base + m], st.o[base:base + m], key)
            got = sh.gather_global(local, base)
            ok.append(bool(got.dtype == np.int32 and np.array_equal(got, orc.match(st.s, st.p, st.o, key))))
        q.put((rank, ok))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gathered_shards_equal_the_whole_store_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ok in got:
        assert all(ok), (rank, ok)


def _rank_that_leaves(rank, world, port, q):
    """Rank 1 leaves before the exchange; rank 0's gather must fail, not hang."""
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_1807_01409_gb300 import shard as sh
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)  # leaves between steps, with nothing in flight
    try:
        sh.gather_global(np.arange(5, dtype=np.int32), 0)
        q.put((rank, "returned"))
    except Exception as e:  # noqa: BLE001 -- the failure is the expected outcome
        q.put((rank, type(e).__name__))


def test_a_rank_that_leaves_fails_the_exchange_gloo():
    """Failure detection on the host: when a rank exits before the shard
    exchange, the remaining rank's collective ends with an error within the
    process group's timeout instead of waiting forever."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_that_leaves, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0
    rank, outcome = q.get(timeout=10)
    assert rank == 0 and outcome != "returned", outcome
