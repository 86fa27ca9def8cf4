"""Benchmark of the TripleID-Q hot path on GB300.

Workload: the university-shaped store (200M triples, int32 SoA columns,
resident in HBM) and its 64 single-pattern queries with selectivity from 1e-6
to 0.3.  One step = every query matched once (scan + compaction of all 64)
through the C ABI.  The metric is triples scanned per second (Gtriples/s),
with the scan kernel's achieved HBM bandwidth against the measured peak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Beside the headline, "rows" times every other row of the path (multi-pattern
scan, bind+filter, sort, joins, union, filter, plan execution) on the same
store, and "batch" times 4096 single-pattern queries on a 500M-triple store
batched (tid_match_batch) against one launch per query on the same GPU, and
"entail" runs the six RDFS rules on the store plus its schema, and
"serve" runs a Poisson request stream through the request server (continuous
batching, admission by estimated bytes) against the same server taking one
request at a time with one search launch per request.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica
of the workload (weak scaling: fixed work per GPU); the step time is the max
over ranks.  --impl reference times the CPU oracle (the plain nested-loop
statement of the method) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1807_01409_gb300 import synth  # noqa: E402

METRIC = "Gtriples/s scanned (% HBM peak); batched/served queries/s + p99 vs plain"
UNIT = "Gtriples/s"
N_TRIPLES = synth.UNI_FULL
WORKLOAD = ("university-200M: 200M triples (int32 SoA, resident), 64 single-pattern "
            "queries, selectivity 1e-6..0.3")
BATCH_TRIPLES = 500_000_000
BATCH_QUERIES = 4096
BATCH_WORKLOAD = ("university-500M (drawn on the device): 500M triples (6 GB int32 SoA, resident), "
                  "4096 single-pattern queries of all seven shapes, result sizes log-uniform 1..1e7")


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (step times: the job ends with its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Work of all ranks over the job's wall time (weak scaling: every rank does units_per_rank)."""
    return units_per_rank * world / seconds


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


K1_REGION = ("// ---- k1_scan: dynamic steps", "int launch_scan(")  # the kernel, its grid and launch


def _kernel_region_sha1(kernel_src):
    src = open(kernel_src).read()
    a, b = src.index(K1_REGION[0]), src.index(K1_REGION[1])
    return hashlib.sha1(src[a:b].encode()).hexdigest()


def _traffic_record(kernel_src):
    """Per-launch DRAM bytes of the scan kernel from the committed ncu record,
    valid only while the kernel's code (its device code, grid and launch) is
    unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "k1_scan_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    try:
        if d.get("kernel_region_sha1") != _kernel_region_sha1(kernel_src):
            return None
    except ValueError:  # the region markers moved: treat as changed
        return None
    return d


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"tid_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle's scan on the host cores
# ---------------------------------------------------------------------------

def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _match_on_cores(orc, store, key, pool, cores):
    """The oracle's match, unchanged, on `cores` contiguous slices of the store at
    once (its C routine runs outside the GIL); the slices' lists, offset by each
    slice's start, concatenate to the ascending list of the whole store."""
    bounds = np.linspace(0, store.n, cores + 1).astype(np.int64)
    parts = list(pool.map(lambda j: orc.match(store.s[bounds[j]:bounds[j + 1]],
                                              store.p[bounds[j]:bounds[j + 1]],
                                              store.o[bounds[j]:bounds[j + 1]], key)
                          + np.int32(bounds[j]),
                          range(cores)))
    return np.concatenate(parts) if parts else np.empty(0, np.int32)


def cpu_baseline(store, queries, budget_s=12.0):
    """The oracle's scan timed on the host: single-threaded (the headline
    baseline), then the same routine over all host cores on contiguous slices."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle
    oracle.build()
    oracle.lib()
    scanned, t0, done = 0, time.perf_counter(), 0
    first = None
    for pat, _, _ in queries:
        r = oracle.match(store.s, store.p, store.o, pat.key())
        if first is None:
            first = r
        scanned += store.n
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    out = {"value": scanned / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{done} of the 64 queries over the full {store.n}-triple store, "
                     f"single-threaded C oracle match ({dt:.1f} s)"}
    cores = _host_cores()
    try:
        with ThreadPoolExecutor(max_workers=cores) as pool:
            got = _match_on_cores(oracle, store, queries[0][0].key(), pool, cores)
            if not np.array_equal(got, first):
                raise RuntimeError("sliced oracle scan differs from the whole-store scan")
            budget_p = budget_s / 2
            scanned_p, done_p, t0 = 0, 0, time.perf_counter()
            for pat, _, _ in queries:
                _match_on_cores(oracle, store, pat.key(), pool, cores)
                scanned_p += store.n
                done_p += 1
                if time.perf_counter() - t0 > budget_p:
                    break
            dtp = time.perf_counter() - t0
        out["all_cores"] = {"value": scanned_p / dtp / 1e9, "unit": UNIT, "cores": cores,
                            "sample": f"{done_p} of the 64 queries over the full store, the same "
                                      f"oracle match on {cores} contiguous slices in {cores} threads "
                                      f"({dtp:.1f} s)"}
    except Exception as e:  # the all-cores figure is context; never lose the line over it
        out["all_cores"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_reference(args, rank, world):
    """The CPU oracle on this workload (rank 0 only)."""
    if rank != 0:
        return
    store = synth.university_store(args.triples)
    queries = synth.university_queries(store)
    from oracle import oracle
    oracle.build()
    per_step = max(1, min(4, len(queries)))  # a bounded sample of each step
    for w in range(args.warmup):
        oracle.match(store.s, store.p, store.o, queries[w % len(queries)][0].key())
    t0 = time.perf_counter()
    scanned = 0
    for k in range(args.steps):
        for j in range(per_step):
            pat = queries[(k * per_step + j) % len(queries)][0]
            oracle.match(store.s, store.p, store.o, pat.key())
            scanned += store.n
    dt = time.perf_counter() - t0
    value = scanned / dt / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD if store.n == N_TRIPLES else
                       f"university-{store.n}: profiling size, not the benchmark workload",
                       "n_triples": store.n, "queries": len(queries),
                       "sample_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} queries per step over the full store"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the other rows of the path, each through the C ABI at full size
# ---------------------------------------------------------------------------

def gather_sectors(idx) -> int:
    """Distinct 32-byte sectors (8 int32) that a gather at these ascending row
    indices touches in one int32 column."""
    sec = np.asarray(idx, np.int64) >> 3
    return 0 if sec.size == 0 else int(np.count_nonzero(np.diff(sec)) + 1)


def measure_rows(tb, ctx, store, st, stream, peak, with_oracle=True, reps=3):
    """Multi-pattern scan, bind (+filter fused), filter, sort (project), join (both
    algorithms), union and plan execution on the university store.  For each:
    GPU time of the C-ABI call (CUDA events on the context stream, best of reps),
    algorithmic bytes (the bytes the operation must move at least: inputs read once,
    outputs written once, plus one read+write pass where the result must be sorted
    -- bind and the reordering projection; joins and unions of canonical inputs
    need none), achieved GB/s against the measured peak, and the oracle's time on
    the same input (or a stated bounded sample)."""
    import torch
    orc = None
    if with_oracle:
        from oracle import oracle as orc
        orc.build()
    n = st.n
    lay = synth.uni_layout(st.meta["subjects"])
    pid, cbase = lay["pred_ids"], lay["class_base"]
    X, Y, Z, V = 0, 1, 2, 4
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    live = []

    def timed(fn):
        best, res = float("inf"), None
        for _ in range(reps):
            if res is not None:
                for h in (res if isinstance(res, list) else [res]):
                    tb.tid_set_free(h)
            torch.cuda.synchronize()
            e0.record(stream)
            res = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        live.extend(res if isinstance(res, list) else [res])
        return best, res

    def rows_of(h):
        return tb.tid_set_rows(h)

    def cpu(fn, scale=1.0):
        if orc is None:
            return None
        t = time.perf_counter()
        fn()
        return (time.perf_counter() - t) * scale * 1e3

    def entry(ms, alg_bytes, cpu_ms, **kw):
        d = {"gpu_ms": round(ms, 4), "algorithmic_bytes": int(alg_bytes),
             "achieved_GBps": round(alg_bytes / (ms / 1e3) / 1e9, 1),
             "frac_of_measured_peak": round(alg_bytes / (ms / 1e3) / 1e9 / peak, 4)}
        if cpu_ms is not None:
            d["oracle_ms"] = round(cpu_ms, 1)
            d["speedup_vs_oracle"] = round(cpu_ms / ms, 1)
        d.update(kw)
        return d

    out = {}
    type_c = synth.Pattern(0, int(pid[0]), int(cbase), var=(X, -1, -1))  # (?x type C), top class 0
    lit = synth.Pattern(0, int(pid[1]), 0, var=(X, -1, V))                 # (?x p1 ?v), literal-valued
    ent = synth.Pattern(0, int(pid[7]), 0, var=(X, -1, Y))                 # (?x p7 ?y), entity-valued

    # a2: one pass for three patterns (union of bound columns: P, O)
    pats = [type_c, lit, ent]
    ms, hs = timed(lambda: tb.tid_match_multi(ctx, store, pats))
    hits = [rows_of(h) for h in hs]
    cpu_ms = cpu(lambda: orc.match_multi(st.s, st.p, st.o, [p.key() for p in pats]))
    out["a2_match_multi"] = entry(ms, 4 * 2 * n + 4 * sum(hits), cpu_ms, patterns=3, hits=hits,
                                  oracle_sample="full store")

    # a3: bind + fused filter from the (?x p1 ?v) index list
    idx = tb.tid_match(ctx, store, lit)
    live.append(idx)
    h = rows_of(idx)
    lo_v, hi_v = synth.LIT_BASE + 10, synth.LIT_BASE + 60
    ms, b = timed(lambda: tb.tid_bind(ctx, store, lit, idx, [(V, "range", lo_v, hi_v)]))
    m = rows_of(b)
    samp = min(h, 2_000_000)
    idx_np = orc.match(st.s, st.p, st.o, lit.key())[:samp] if orc else None
    cpu_ms = cpu(lambda: orc.filter(orc.bind(st.s, st.p, st.o, lit.key(), lit.var, idx_np), V, "range",
                                    lo_v, hi_v), scale=h / samp) if orc else None
    out["a3_bind_filter"] = entry(ms, 4 * h + 8 * h + 8 * m + 16 * m, cpu_ms, rows_in=h, rows_out=m,
                                  oracle_sample=f"first {samp} indices, time scaled x{h / samp:.1f}")
    # the gathers move whole 32-byte sectors: the least DRAM traffic they can cause
    sect = gather_sectors(tb.tid_set_to_host(idx)[:, 0])
    sb = 2 * 32 * sect + 4 * h + 8 * m + 16 * m
    out["a3_bind_filter"].update({"sector_bytes": int(sb), "gathered_sectors_per_column": sect,
                                  "frac_of_measured_peak_sector_bytes": round(sb / (ms / 1e3) / 1e9 / peak, 4)})

    # a4: filter on a bound set (x, v) of all (?x p1 ?v)
    full = tb.tid_bind(ctx, store, lit, idx, [])
    live.append(full)
    nf = rows_of(full)
    ms, f = timed(lambda: tb.tid_filter(ctx, full, [(V, "range", lo_v, hi_v)]))
    mf = rows_of(f)
    samp = min(nf, 4_000_000)
    sample_set = orc.TupleSet((X, V), tb.tid_set_to_host(full)[:samp]) if orc else None
    cpu_ms = cpu(lambda: orc.filter(sample_set, V, "range", lo_v, hi_v), scale=nf / samp) if orc else None
    out["a4_filter"] = entry(ms, 8 * nf + 8 * mf, cpu_ms, rows_in=nf, rows_out=mf,
                             oracle_sample=f"first {samp} rows, time scaled x{nf / samp:.1f}")

    # a5/a8: sort = project (x, v) -> (v, x) with DISTINCT: a full canonical sort
    ms, pr = timed(lambda: tb.tid_project(ctx, full, (V, X)))
    mp = rows_of(pr)
    cpu_ms = cpu(lambda: orc.project(sample_set, (V, X)), scale=nf / samp) if orc else None
    out["a5_a8_sort_project"] = entry(ms, 8 * nf + 8 * mp + 16 * mp, cpu_ms, rows_in=nf, rows_out=mp,
                                      oracle_sample=f"first {samp} rows, time scaled x{nf / samp:.1f}")

    # a6: join (?x type C)(x) with (?x p7 ?y)(x, y) on x, both algorithms
    it = tb.tid_match(ctx, store, type_c)
    ie = tb.tid_match(ctx, store, ent)
    live += [it, ie]
    L = tb.tid_bind(ctx, store, type_c, it, [])
    R = tb.tid_bind(ctx, store, ent, ie, [])
    live += [L, R]
    nl, nr = rows_of(L), rows_of(R)
    Lh, Rh = (tb.tid_set_to_host(L), tb.tid_set_to_host(R)) if orc else (None, None)
    cpu_join = cpu(lambda: orc.join(orc.TupleSet((X,), Lh), orc.TupleSet((X, Y), Rh), method="sortmerge"))
    for algo in ("sort_merge", "hash"):
        ms, j = timed(lambda: tb.tid_join(ctx, L, R, algo))
        mj = rows_of(j)
        cpu_ms = cpu_join
        out[f"a6_join_{algo}"] = entry(ms, 4 * nl + 8 * nr + 8 * mj, cpu_ms, rows_l=nl, rows_r=nr,
                                       rows_out=mj, oracle_sample="full inputs (oracle sort-merge join)")

    # the outer joins on the same inputs: left (OPTIONAL), and right and full composed from it;
    # algorithmic bytes: both inputs read once, the output written once
    sl, sr = min(nl, 50_000), min(nr, 400_000)
    if orc:
        Ls_, Rs_ = orc.TupleSet((X,), Lh[:sl]), orc.TupleSet((X, Y), Rh[:sr])
    for kind in ("left", "right", "full"):
        try:
            ms, j = timed(lambda: tb.tid_join(ctx, L, R, kind))
            mj = rows_of(j)
            cpu_ms = cpu(lambda: getattr(orc, f"{kind}_join")(Ls_, Rs_), scale=(nl + nr) / max(1, sl + sr)) \
                if orc else None
            out[f"outer_join_{kind}"] = entry(ms, 4 * nl + 8 * nr + 8 * mj, cpu_ms, rows_l=nl, rows_r=nr, rows_out=mj,
                                              oracle_sample=f"first {sl} and {sr} rows of the inputs, time scaled "
                                                            f"x{(nl + nr) / max(1, sl + sr):.1f}")
        except Exception as e:  # noqa: BLE001 -- reported in the line
            out[f"outer_join_{kind}"] = {"error": f"{type(e).__name__}: {e}"}

    # a7: union of (x, v) and (x, y): schema (x, v, y), padded with 0
    ms, u = timed(lambda: tb.tid_union(ctx, [full, R]))
    mu = rows_of(u)
    cpu_ms = None
    if orc:
        su = min(samp, nr)
        a_s = orc.TupleSet((X, V), tb.tid_set_to_host(full)[:su])
        b_s = orc.TupleSet((X, Y), Rh[:su])
        cpu_ms = cpu(lambda: orc.union([a_s, b_s]), scale=(nf + nr) / (2 * su))
    out["a7_union"] = entry(ms, 8 * nf + 8 * nr + 12 * mu, cpu_ms, rows_in=nf + nr,
                            rows_out=mu, oracle_sample="bounded sample of both inputs, time scaled")
    for h_ in live:
        tb.tid_set_free(h_)
    live.clear()

    # a9: the 48 plans (star, chain, union, filter) through tid_exec
    plans = synth.university_plans(st)
    lat = []
    for name, plan in plans:  # warm-up
        h_ = tb.tid_exec(ctx, store, plan)
        rows_of(h_)
        tb.tid_set_free(h_)
    for r in range(reps):
        for name, plan in plans:
            torch.cuda.synchronize()
            t = time.perf_counter()
            h_ = tb.tid_exec(ctx, store, plan)
            rows_of(h_)
            lat.append((time.perf_counter() - t) * 1e3)
            tb.tid_set_free(h_)
    lat = np.array(lat)
    cpu_ms = None
    sample_names = ("filter5", "union3", "star11")
    if orc:
        t = time.perf_counter()
        for name, plan in plans:
            if name in sample_names:
                orc.execute(st.s, st.p, st.o, plan)
        cpu_ms = (time.perf_counter() - t) * 1e3 / len(sample_names)
    out["a9_exec"] = {"plans": len(plans), "queries_per_s": round(len(lat) / (lat.sum() / 1e3), 1),
                      "latency_ms_p50": round(float(np.percentile(lat, 50)), 3),
                      "latency_ms_p99": round(float(np.percentile(lat, 99)), 3),
                      "oracle_ms_per_plan": None if cpu_ms is None else round(cpu_ms, 1),
                      "oracle_sample": f"plans {', '.join(sample_names)}, full store"}
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist

    from paper_1807_01409_gb300 import binding as tb
    from paper_1807_01409_gb300 import build as tbuild

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tbuild.build()

    store_np = synth.university_store(args.triples)
    queries = [q for q, _, _ in synth.university_queries(store_np, seed=synth.QUERY_SEED + rank)]
    nq = len(queries)
    bound = [sum(1 for x in q.key() if x != 0) for q in queries]

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = tb.tid_ctx_create(local, stream.cuda_stream)
    cols = [torch.from_numpy(c).cuda() for c in (store_np.s, store_np.p, store_np.o)]
    torch.cuda.synchronize()
    store = tb.tid_load(ctx, *cols, copy=0)

    def step(events=None):
        hs = []
        for j, q in enumerate(queries):
            if events is not None:
                events[j][0].record(stream)
            hs.append(tb.tid_match(ctx, store, q))
            if events is not None:
                events[j][1].record(stream)
        rows = [tb.tid_set_rows(h) for h in hs]
        for h in hs:
            tb.tid_set_free(h)
        return rows

    for _ in range(args.warmup):
        rows = step()
    hits = rows

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nq)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with Clocks(local) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            step(ev[k])
        t_end.record(stream)
        barrier()
    ms = max_over_ranks(t_start.elapsed_time(t_end), world, "cuda")
    kernel_ms = [ev[k][j][0].elapsed_time(ev[k][j][1]) for k in range(args.steps) for j in range(nq)]
    step_stats = step_span_stats(ev)
    total_kernel_ms = sum(kernel_ms)
    alg_bytes_step = sum(4 * b * store_np.n + 4 * h for b, h in zip(bound, hits))
    scanned_step = nq * store_np.n
    value = whole_job_rate(scanned_step * args.steps, world, ms / 1e3) / 1e9

    peak, peak_kind = _peaks()
    achieved = alg_bytes_step * args.steps / (total_kernel_ms / 1e3) / 1e9
    tr = _traffic_record(os.path.join(ROOT, "paper_1807_01409_gb300", "csrc", "match.cu"))
    traffic = None
    if tr is not None:
        traffic = tr.get("dram_bytes_per_launch")

    # ------------------------------------------------------------------ e2e
    # host buffers: the store is copied in from pinned memory and every result
    # list copied back into pinned memory, each step, through the public C ABI
    host_cols = [torch.from_numpy(c).pin_memory() for c in (store_np.s, store_np.p, store_np.o)]
    e2e_steps = max(1, args.steps)  # as many steps as the device-timed value
    out_bufs = [torch.empty((max(h, 1), 1), dtype=torch.int32).pin_memory().numpy() for h in hits]
    d2h = 4 * sum(hits)
    h2d = 3 * 4 * store_np.n

    def e2e_step():
        st = tb.tid_load(ctx, *host_cols, where=tb.TID_HOST)
        hs = [tb.tid_match(ctx, st, q) for q in queries]
        for h, buf in zip(hs, out_bufs):
            tb.tid_set_to_host(h, buf)
            tb.tid_set_free(h)
        tb.tid_store_free(st)

    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    e2e_value = whole_job_rate(scanned_step * e2e_steps, world, e2e_s) / 1e9

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(store_np, synth.university_queries(store_np))
    # the other rows are per-GPU characteristics: measured in single-GPU runs only;
    # a row that fails reports its error and the line is printed all the same
    extra = world == 1
    oracle_too = rank == 0 and world == 1 and not args.no_cpu_baseline
    rows = None
    if extra and not args.no_rows:
        rows = _row(lambda: measure_rows(tb, ctx, store, store_np, stream, _peaks()[0], with_oracle=oracle_too))

    tb.tid_store_free(store)
    del cols
    torch.cuda.empty_cache()
    entail = None
    if extra and not args.no_entail:
        entail = _row(lambda: measure_entail(tb, ctx, stream, store_np, _peaks()[0], with_oracle=oracle_too))
    batch = None
    if extra and not args.no_batch:
        batch = _row(lambda: measure_batch(tb, ctx, stream, _peaks()[0], with_oracle=oracle_too))
    _row(lambda: tb.tid_ctx_destroy(ctx))
    serve = None
    if extra and not args.no_serve:
        serve = _row(lambda: measure_serve(tb, with_oracle=oracle_too))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "step_ms": step_stats,
            "config": {"workload": WORKLOAD if store_np.n == N_TRIPLES else
                       f"university-{store_np.n}: profiling size, not the benchmark workload",
                       "n_triples": store_np.n, "queries": nq,
                       "hits_per_step": int(sum(hits)),
                       "l2": "inputs larger than L2 (every scan reads >= 800 MB)",
                       "parallelism": f"replica x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "frac_of_8TBs_nominal": achieved / 8000.0,
                         "traffic": traffic, "kernel": "k1_scan",
                         "algorithmic_bytes_per_step": alg_bytes_step,
                         "avg_launch_us": total_kernel_ms * 1e3 / len(kernel_ms)},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps},
            "gpu_launches": nq * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": base,
            "rows": rows,
            "entail": entail,
            "batch": batch,
            "serve": serve,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _row(fn):
    """fn()'s result, or {"error": ...} if it raises."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 -- reported in the JSON line
        return {"error": f"{type(e).__name__}: {e}"}


def step_span_stats(ev):
    """Best and median step time (ms, this rank) from per-launch event pairs
    ev[step][launch] = (start, end): a step spans its first launch's start to its
    last launch's end."""
    spans = [steps[0][0].elapsed_time(steps[-1][1]) for steps in ev if steps]
    if not spans:
        return None
    return {"best": min(spans), "median": statistics.median(spans), "steps": len(spans)}


def _pct(x, q):
    return float(np.percentile(np.asarray(x, np.float64), q))


def measure_batch(tb, ctx, stream, peak, n=BATCH_TRIPLES, m=BATCH_QUERIES, with_oracle=True, reps=24):
    """Batched search against one launch per query on the same GPU: 4096 patterns
    over a 500M-triple store.  Batched: one tid_match_batch call (every query is
    answered when it returns).  Plain: one tid_match per query in submission order
    (a query's latency is the time from the start to its own scan's completion).
    Both from the same start, all queries submitted at once."""
    import torch

    s, p, o = synth.university_store_torch(n, device="cuda")
    qs = synth.batch_queries(s, p, o, m=m)
    keys = np.array([q.key() for q, _, _ in qs], np.int64)
    pats = tb.pattern_array(keys)
    sizes = np.array([sz for _, _, sz in qs], np.int64)
    distinct = {}
    for pat, _, sz in qs:
        distinct[pat.key()] = sz
    dk = list(distinct)
    alg_bytes = 0
    for b in range(0, len(dk), tb.TID_BATCH_KEYS):  # per sub-batch: two passes over its columns
        cols = 0
        for k in dk[b:b + tb.TID_BATCH_KEYS]:
            cols |= sum(1 << j for j in range(3) if k[j])
        alg_bytes += 2 * 4 * bin(cols).count("1") * n
    alg_bytes += 4 * sum(distinct.values())
    torch.cuda.synchronize()
    store = tb.tid_load(ctx, s, p, o, copy=0)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    for h in tb.tid_match_batch(ctx, store, pats):
        tb.tid_set_free(h)
    tuning = tb.tid_batch_tuning(ctx)
    batch_ms, hits_ok = [], True
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        hs = tb.tid_match_batch(ctx, store, pats)
        e1.record(stream)
        e1.synchronize()
        batch_ms.append(e0.elapsed_time(e1))
        got = np.array([tb.tid_set_rows(h) for h in hs], np.int64)
        hits_ok = hits_ok and bool(np.array_equal(got, sizes))
        for h in hs:
            tb.tid_set_free(h)

    two = _two_pattern_batch(tb, s, p, o)

    plist = [tb.as_pattern(tuple(int(x) for x in k)) for k in keys]
    for q in plist[:64]:
        tb.tid_set_free(tb.tid_match(ctx, store, q))
    torch.cuda.synchronize()
    done = [ev() for _ in plist]
    e0, e1 = ev(), ev()
    e0.record(stream)
    for q, e in zip(plist, done):
        h = tb.tid_match(ctx, store, q)
        e.record(stream)
        tb.tid_set_free(h)
    e1.record(stream)
    e1.synchronize()
    plain_ms = e0.elapsed_time(e1)
    plain_lat = [e0.elapsed_time(e) for e in done]
    tb.tid_store_free(store)

    oracle = None
    if with_oracle:
        from oracle import oracle as orc
        orc.build()
        hs_, hp_, ho_ = (t.cpu().numpy() for t in (s, p, o))
        t0, cnt = time.perf_counter(), 0
        for k in keys[:: max(1, m // 64)]:
            orc.match(hs_, hp_, ho_, tuple(int(x) for x in k))
            cnt += 1
            if time.perf_counter() - t0 > 10.0:
                break
        dt = time.perf_counter() - t0
        oracle = {"value": cnt / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
                  "sample": f"{cnt} of the {m} queries (every {max(1, m // 64)}th), each a full "
                            f"single-threaded C oracle scan of the {n}-triple store ({dt:.1f} s)"}
        del hs_, hp_, ho_
    del s, p, o
    torch.cuda.empty_cache()
    bms = statistics.median(batch_ms)
    return {
        "workload": BATCH_WORKLOAD if n == BATCH_TRIPLES else f"university-{n}: profiling size, not the "
                                                              f"batched workload",
        "n_triples": n, "queries": m, "distinct_keys": len(dk),
        "sub_batches": (len(dk) + tb.TID_BATCH_KEYS - 1) // tb.TID_BATCH_KEYS,
        "result_rows": int(sizes.sum()), "result_rows_distinct_keys": int(sum(distinct.values())),
        "results_match_tallies": hits_ok,
        "autotuner": tuning,
        "batched": {"ms": bms, "calls": len(batch_ms), "ms_all": [round(x, 3) for x in batch_ms],
                    "queries_per_s": m / (bms / 1e3),
                    "p50_ms": _pct(batch_ms, 50), "p99_ms": _pct(batch_ms, 99),
                    "latency": "a batched query is answered when its call returns: its latency is the "
                               "call's duration; p50/p99 over the calls"},
        "plain": {"ms": plain_ms, "queries_per_s": m / (plain_ms / 1e3),
                  "p50_ms": _pct(plain_lat, 50), "p99_ms": _pct(plain_lat, 99)},
        "speedup_queries_per_s": plain_ms / bms,
        "p99_ratio_plain_over_batched": _pct(plain_lat, 99) / _pct(batch_ms, 99),
        "hbm": {"algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / (bms / 1e3) / 1e9,
                "frac_of_peak": alg_bytes / (bms / 1e3) / 1e9 / peak,
                "note": "whole call: both passes of every sub-batch, the scans of counts, the "
                        "host synchronisation between passes and set creation"},
        "cpu_baseline": oracle,
        "two_pattern": two,
    }


def _two_pattern_batch(tb, s, p, o, m=1024):
    """Two-pattern queries (star joins of two bound (predicate, object) pairs of one
    subject), all arriving at once, through the request server: batched (one search
    for the wave, then each join) against one request at a time, each searching alone."""
    kinds, plans, _ = synth.serving_requests(s, p, o, m=m, seed=synth.QUERY_SEED + 4096, mix=(0.0, 1.0, 0.0))
    prepared = [tb.Server.request(k, x) for k, x in zip(kinds, plans)]
    out = {"queries": m, "shape": "(?x p1 o1) JOIN (?x p2 o2)"}
    for name, kw in (("batched", dict(workers=2, max_wave=4096, batch_scans=True)),
                     ("plain", dict(workers=1, max_wave=1, batch_scans=False))):
        with tb.Server(s, p, o, budget_bytes=SERVE_BUDGET, **kw) as srv:
            for rid in [srv.submit(x) for x in prepared[:16]]:
                srv.wait(rid)
                srv.release(rid)
            t0 = tb.Server.now_ns()
            ids = [srv.submit(x, t0) for x in prepared]
            lat = []
            for rid in ids:
                srv.wait(rid)
                lat.append(srv.result(rid)[3] / 1e6)
            span = max(lat) / 1e3
        out[name] = {"ms": span * 1e3, "queries_per_s": m / span, "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99)}
    out["speedup_queries_per_s"] = out["batched"]["queries_per_s"] / out["plain"]["queries_per_s"]
    return out


def measure_entail(tb, ctx, stream, store_np, peak, with_oracle=True, oracle_n=20_000_000):
    """The six RDFS rules (tid_entail) on the university store plus its schema:
    per rule the call's time (CUDA events; the call synchronises), the paper's step
    counts, and the algorithmic bytes of its two store passes over that time: the
    schema search reads P (4n), the keyed search reads P for every triple (the fixed
    predicate or the key itself, 4n) and the other columns of the triples it keeps
    (at most 8 bytes each of res2).  The oracle runs the same rules on a smaller store
    of the same recipe, beside the GPU on that store."""
    import torch

    def run(st_np):
        vocab = synth.rdfs_vocab(st_np.meta["subjects"])
        cols = [torch.from_numpy(c).cuda() for c in (st_np.s, st_np.p, st_np.o)]
        torch.cuda.synchronize()
        st = tb.tid_load(ctx, *cols, copy=0)
        res = {}
        for rule in tb.RULES:
            h, _ = tb.tid_entail(ctx, st, rule, vocab)  # warm-up
            tb.tid_set_free(h)
            ms = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h, stats = tb.tid_entail(ctx, st, rule, vocab)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                tb.tid_set_free(h)
            t = statistics.median(ms)
            scan_bytes = 8 * st_np.n + 8 * stats["res2"]
            res[f"R{rule}"] = {"gpu_ms": round(t, 3), **stats,
                               "store_pass_bytes": scan_bytes,
                               "store_pass_GBps": round(scan_bytes / (t / 1e3) / 1e9, 1),
                               "frac_of_measured_peak": round(scan_bytes / (t / 1e3) / 1e9 / peak, 4)}
        tb.tid_store_free(st)
        del cols
        return res, vocab

    full = synth.with_schema(store_np)
    out = {"workload": f"university-{store_np.n} + its RDFS schema ({full.meta['schema_triples']} triples)",
           "rules": run(full)[0]}
    if with_oracle:
        from oracle import oracle as orc
        orc.build()
        small = synth.with_schema(synth.university_store(oracle_n))
        g_small, vocab = run(small)
        cmp_ = {}
        for rule in tb.RULES:
            t0 = time.perf_counter()
            orc.entail(small.s, small.p, small.o, rule, vocab)
            cmp_[f"R{rule}"] = {"oracle_ms": round((time.perf_counter() - t0) * 1e3, 1),
                                "gpu_ms": g_small[f"R{rule}"]["gpu_ms"]}
            cmp_[f"R{rule}"]["speedup_vs_oracle"] = round(cmp_[f"R{rule}"]["oracle_ms"] /
                                                          max(cmp_[f"R{rule}"]["gpu_ms"], 1e-6), 1)
        out["oracle_comparison"] = {"n_triples": small.n, "cores": 1, "kind": "oracle", "rules": cmp_}
    torch.cuda.empty_cache()
    return out


SERVE_TRIPLES = 1_000_000_000
SERVE_REQUESTS = 4000
SERVE_RATE = 20000.0
SERVE_BUDGET = 60 << 30
SERVE_WORKLOAD = ("university-1B (drawn on the device): 1B triples (12 GB int32 SoA, resident), Poisson "
                  "arrivals at 20k requests/s: 68% index lookups (result sizes log-uniform 1..1e5), 14% "
                  "two-pattern star joins, 14% unions / literal-range filters, 2% wide scans (result sizes "
                  "log-uniform 1e5..0.3n), 2% typed star joins (intermediates of 0.1-20M rows); 60 GB "
                  "admission budget")


def _serve_stream(tb, srv, prepared, arrivals):
    """Submit every request at its arrival time (open loop), wait for all; latencies
    run from the scheduled arrival."""
    t0 = tb.Server.now_ns() + 20_000_000
    due = (t0 + np.asarray(arrivals) * 1e9).astype(np.int64)
    ids, i, m = [], 0, len(prepared)
    while i < m:
        now = tb.Server.now_ns()
        while i < m and due[i] <= now:
            ids.append(srv.submit(prepared[i], int(due[i])))
            i += 1
        if i < m:
            time.sleep(max(0.0, min(1e-3, (due[i] - tb.Server.now_ns()) / 1e9)))
    lat, fin, bad = [], [], 0
    for rid, d in zip(ids, due):
        srv.wait(rid)
        st, _, rows, ln = srv.result(rid)
        bad += st != tb.TID_OK
        lat.append(ln / 1e6)
        fin.append(int(d) + ln)
    span = (max(fin) - t0) / 1e9
    return {"requests": m, "seconds": span, "queries_per_s": m / span, "p50_ms": _pct(lat, 50),
            "p99_ms": _pct(lat, 99), "max_ms": max(lat), "failed": int(bad)}


def measure_serve(tb, n=SERVE_TRIPLES, m=SERVE_REQUESTS, rate=SERVE_RATE, with_oracle=True):
    """The request server against the same server run one request at a time with one
    search launch per request, on the same Poisson stream."""
    import torch

    s, p, o = synth.university_store_torch(n, device="cuda")
    kinds, payloads, arrivals = synth.serving_requests(s, p, o, m=m, rate=rate)
    prepared = [tb.Server.request(k, x) for k, x in zip(kinds, payloads)]
    torch.cuda.synchronize()
    out = {"workload": SERVE_WORKLOAD, "n_triples": n, "offered_queries_per_s": rate,
           "mix": {k: kinds.count(k) for k in set(kinds)}}
    for name, kw in (("served", dict(workers=2, max_wave=4096, batch_scans=True, budget_bytes=SERVE_BUDGET)),
                     ("plain", dict(workers=1, max_wave=1, batch_scans=False, budget_bytes=SERVE_BUDGET))):
        with tb.Server(s, p, o, **kw) as srv:
            warm = [srv.submit(x) for x in prepared[:32]]
            for rid in warm:
                srv.wait(rid)
                srv.release(rid)
            res = _serve_stream(tb, srv, prepared, arrivals)
            res["stats"] = srv.stats()
            res["config"] = kw
        out[name] = res
    out["speedup_queries_per_s"] = out["served"]["queries_per_s"] / out["plain"]["queries_per_s"]
    out["p99_ratio_plain_over_served"] = out["plain"]["p99_ms"] / out["served"]["p99_ms"]
    if with_oracle:
        from oracle import oracle as orc
        orc.build()
        hs_, hp_, ho_ = (t.cpu().numpy() for t in (s, p, o))
        t0, cnt = time.perf_counter(), 0
        for k, x in zip(kinds, payloads):
            if k == "index":
                orc.match(hs_, hp_, ho_, x.key())
            else:
                orc.execute(hs_, hp_, ho_, x)
            cnt += 1
            if time.perf_counter() - t0 > 10.0:
                break
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": cnt / dt, "unit": "queries/s", "cores": 1, "kind": "oracle",
                               "sample": f"the first {cnt} requests of the stream, one after another, "
                                         f"single-threaded oracle on the {n}-triple store ({dt:.1f} s)"}
        del hs_, hp_, ho_
    del s, p, o
    torch.cuda.empty_cache()
    return out


def run_serve_only(args, local):
    """One served-versus-plain measurement (no oracle), for launch-list captures."""
    import torch

    from paper_1807_01409_gb300 import binding as tb
    from paper_1807_01409_gb300 import build as tbuild
    torch.cuda.set_device(local)
    tbuild.build()
    print(json.dumps({"serve": measure_serve(tb, with_oracle=False)}), flush=True)


def run_batch_only(args, local):
    """One batched-versus-plain measurement (no oracle), for launch-list captures."""
    import torch

    from paper_1807_01409_gb300 import binding as tb
    from paper_1807_01409_gb300 import build as tbuild
    torch.cuda.set_device(local)
    tbuild.build()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = tb.tid_ctx_create(local, stream.cuda_stream)
    res = measure_batch(tb, ctx, stream, _peaks()[0], n=args.batch_triples, with_oracle=False, reps=1)
    tb.tid_ctx_destroy(ctx)
    print(json.dumps({"batch": res}), flush=True)


def run_rows_only(args, local):
    """One pass of measure_rows on the university store (no oracle), for launch-list captures."""
    import torch

    from paper_1807_01409_gb300 import binding as tb
    from paper_1807_01409_gb300 import build as tbuild
    torch.cuda.set_device(local)
    tbuild.build()
    st = synth.university_store(args.triples)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = tb.tid_ctx_create(local, stream.cuda_stream)
    cols = [torch.from_numpy(c).cuda() for c in (st.s, st.p, st.o)]
    torch.cuda.synchronize()
    store = tb.tid_load(ctx, *cols, copy=0)
    rows = measure_rows(tb, ctx, store, st, stream, _peaks()[0], with_oracle=False, reps=args.rows_reps)
    tb.tid_store_free(store)
    tb.tid_ctx_destroy(ctx)
    print(json.dumps({"rows": rows, "n_triples": st.n}), flush=True)


def run_sort_only(args, local):
    """The canonical sort alone, for profiling: a seeded three-column set of
    n rows (a 20-bit leading column, then a 23-bit and a 12-bit one), made
    canonical by tid_set_from_host, then projected onto its last two columns
    (35-bit packed keys: pack, five digit passes, distinct rows kept), timed
    with CUDA events on the context's stream.  The same again with a 3-bit last
    column (26-bit keys, four passes)."""
    import numpy as np
    import torch

    from paper_1807_01409_gb300 import binding as tb
    from paper_1807_01409_gb300 import build as tbuild
    torch.cuda.set_device(local)
    tbuild.build()
    n, reps = args.sort_only, max(1, args.rows_reps)
    rng = np.random.default_rng(synth.QUERY_SEED)
    stream = torch.cuda.Stream()
    ctx = tb.tid_ctx_create(local, stream.cuda_stream)
    res = {}
    for name, c1, c2 in [("35bit", rng.integers(1, 5_000_000, n), 5_000_001 + 512 * rng.integers(0, 8, n)),
                         ("26bit", rng.integers(1, 5_000_000, n), rng.integers(0, 8, n))]:
        rows = np.stack([rng.integers(1, 1 << 20, n), c1, c2], 1).astype(np.int32)
        S = tb.tid_set_from_host(ctx, rows, [0, 1, 2])
        tb.tid_ctx_sync(ctx)
        ts = []
        for _ in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            P = tb.tid_project(ctx, S, [1, 2])
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
            out_rows = tb.tid_set_rows(P)
            tb.tid_set_free(P)
        tb.tid_set_free(S)
        timed = sorted(ts[2:])
        res[name] = {"rows_in": n, "rows_out": out_rows, "ms_median": round(timed[len(timed) // 2], 4),
                     "ms_all": [round(t, 4) for t in ts]}
    tb.tid_ctx_destroy(ctx)
    print(json.dumps({"sort": res}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the other rows of the path")
    ap.add_argument("--rows-only", action="store_true",
                    help="profiling aid: one pass of the other rows only (no oracle), printed as JSON")
    ap.add_argument("--rows-reps", type=int, default=1,
                    help="with --rows-only: calls per row (best of; 1 for launch-list captures)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-queries row")
    ap.add_argument("--batch-only", action="store_true",
                    help="profiling aid: one batched-versus-plain measurement only, printed as JSON")
    ap.add_argument("--batch-triples", type=int, default=BATCH_TRIPLES,
                    help="store size of --batch-only (default: the 500M workload; smaller only for profiling)")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-requests row")
    ap.add_argument("--no-entail", action="store_true", help="skip the RDFS entailment row")
    ap.add_argument("--serve-only", action="store_true",
                    help="profiling aid: one served-versus-plain measurement only, printed as JSON")
    ap.add_argument("--sort-only", type=int, default=0, metavar="N",
                    help="time the canonical sort of N seeded rows alone (calls: --rows-reps) and exit")
    ap.add_argument("--triples", type=int, default=N_TRIPLES,
                    help="store size (default: the full 200M workload; smaller only for profiling)")
    args = ap.parse_args()
    rank, world, local = _env_rank()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.sort_only:
        run_sort_only(args, local)
    elif args.rows_only:
        run_rows_only(args, local)
    elif args.batch_only:
        run_batch_only(args, local)
    elif args.serve_only:
        run_serve_only(args, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
