"""The multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): the
step time is the maximum over ranks, the value is the work of all ranks over
that time, and the reference arm prints from rank 0 only."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # rank 1 is slower
        rate = bench.whole_job_rate(64 * 200e6, world, ms / 1e3)
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in got:
        assert ms == 15.0                      # the slowest rank
        assert rate == pytest.approx(2 * 64 * 200e6 / 0.015)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(100.0, 1, 2.0) == 50.0


def test_reference_arm_prints_on_rank0_only(tmp_path):
    """Under a launcher, a rank other than 0 exits 0 without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_all_cores_oracle_scan_equals_whole_store_scan():
    """The all-cores CPU baseline runs the oracle's match on contiguous slices;
    offset and concatenated, the slices give the whole store's list, including
    slice counts that leave empty or one-triple slices."""
    from concurrent.futures import ThreadPoolExecutor
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle
    from paper_1807_01409_gb300 import synth
    st = synth.university_store(50_000)
    keys = [q.key() for q, _, _ in synth.university_queries(st)[:8]] + [(0, 0, 0)]
    with ThreadPoolExecutor(max_workers=4) as pool:
        for cores in (1, 3, 7, 64):
            for key in keys:
                want = oracle.match(st.s, st.p, st.o, key)
                got = bench._match_on_cores(oracle, st, key, pool, cores)
                assert got.dtype == want.dtype and np.array_equal(got, want), (cores, key)
    tiny = synth.Store(st.s[:3].copy(), st.p[:3].copy(), st.o[:3].copy(), "tiny")
    with ThreadPoolExecutor(max_workers=2) as pool:
        assert np.array_equal(bench._match_on_cores(oracle, tiny, (0, 0, 0), pool, 8),
                              np.arange(3, dtype=np.int32))


def test_step_span_stats():
    """Per-step spans from (start, end) event pairs: first start to last end."""
    sys.path.insert(0, ROOT)
    import bench

    class Ev:
        def __init__(self, t):
            self.t = t

        def elapsed_time(self, other):
            return other.t - self.t

    ev = [[(Ev(0.0), Ev(1.0)), (Ev(1.5), Ev(4.0))],
          [(Ev(10.0), Ev(11.0)), (Ev(11.0), Ev(13.0))],
          [(Ev(20.0), Ev(20.5)), (Ev(21.0), Ev(26.0))]]
    st = bench.step_span_stats(ev)
    assert st == {"best": 3.0, "median": 4.0, "steps": 3}
    assert bench.step_span_stats([]) is None


def test_traffic_record_follows_the_kernel_source(tmp_path):
    """The committed DRAM-traffic record is used only while the scan kernel's
    source (its section of match.cu) is the one it was captured on."""
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_1807_01409_gb300", "csrc", "match.cu")
    text = open(src).read()
    rec = bench._traffic_record(src)
    if rec is not None:  # recorded on this kernel: the region hash matches
        assert rec["kernel_region_sha1"] == bench._kernel_region_sha1(src)
    outside = tmp_path / "outside.cu"  # an edit outside the kernel's section keeps the record
    outside.write_text("// host-side note\n" + text)
    assert (bench._traffic_record(str(outside)) is None) == (rec is None)
    a = text.index(bench.K1_REGION[0]) + len(bench.K1_REGION[0])
    inside = tmp_path / "inside.cu"  # an edit inside it drops the record
    inside.write_text(text[:a] + "\n// changed\n" + text[a:])
    assert bench._traffic_record(str(inside)) is None
    gone = tmp_path / "gone.cu"  # section markers missing: no record
    gone.write_text(text.replace(bench.K1_REGION[0], ""))
    assert bench._traffic_record(str(gone)) is None


def test_gather_sectors():
    """Sectors of 8 int32 touched by a gather at ascending indices."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.gather_sectors(np.array([], np.int32)) == 0
    assert bench.gather_sectors(np.array([0, 1, 7], np.int32)) == 1
    assert bench.gather_sectors(np.array([7, 8], np.int32)) == 2
    assert bench.gather_sectors(np.array([0, 16, 17, 40, 2 ** 31 - 1], np.int32)) == 4
    idx = np.sort(np.random.default_rng(3).choice(10_000, 3000, replace=False)).astype(np.int32)
    assert bench.gather_sectors(idx) == np.unique(idx // 8).size


def test_failed_row_is_reported_not_raised():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._row(lambda: {"a": 1}) == {"a": 1}

    def boom():
        raise RuntimeError("no device")
    assert bench._row(boom) == {"error": "RuntimeError: no device"}
