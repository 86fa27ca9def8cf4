"""Seeded synthetic TripleID stores and query workloads.

This module only draws inputs: dictionary-encoded int32 triple columns in
structure-of-arrays layout and the triple patterns / plans asked of them.  It
holds none of the query method's arithmetic (no pattern matching, joining or
compaction); both the CPU oracle and the CUDA library consume what it makes.

ID space (one shared namespace, so a subject ID and an object ID that are equal
denote the same term -- the worked example of the entailment section joins
object 56 with subject 56):

* 0 is reserved for the free variable "?" (Section 3, the key encoding);
* entity IDs lie in [1, 2^30 - 1];
* an encoded integer literal of value v in [0, 2^30 - 1] has ID LIT_BASE + v,
  LIT_BASE = 2^30, so ID order equals value order (the order-preserving ID
  assignment suggested in Section 4.3).

Workloads (the paper's BTC-2009 and SP2Bench files are not available; these
stand in for them with the same kind of skew):

* ``tiny``       -- 1M triples; S uniform over 1..100k, P = Zipf(1.2) rank over
                    1..64, O = Zipf(1.1) rank over 1..200k; 16 queries, 4 each of
                    (s,?,?), (?,p,?), (?,p,o), (s,p,?) keyed from stored triples.
* ``university`` -- a university-shaped ontology (20 predicates with fixed
                    frequencies, typed subject classes, 60% entity-valued and
                    40% literal-valued objects); 200M triples at full size, any
                    smaller size for parity runs; 64 single-pattern queries with
                    target selectivity log-uniform on [1e-6, 0.3]; plans of
                    star and chain joins, unions and literal-range filters.
* ``university_store_torch`` -- the same recipe drawn on the GPU with torch
                    (500M / 1B triples in seconds; other values than the host
                    generator's), for the batched and the serving workloads.
* ``batch_queries`` -- 4096 single-pattern queries of all seven bound-position
                    shapes with result sizes log-uniform on [1, 1e7].
* ``serving_requests`` -- a Poisson request stream (index lookups, two-pattern
                    star joins, unions and filters) with arrival times.
* ``rdfs_schema`` -- an RDFS schema over the university classes and predicates
                    (subClassOf trees, domain/range, subPropertyOf chains) for
                    the entailment rules of Section 5.

Every store is a set: duplicate triples are removed and the store topped up to
exactly ``n`` triples, then put in a seeded random order (the store is neither
sorted nor indexed, as in the paper).
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass, field

import numpy as np

LIT_BASE = 1 << 30
STORE_SEED = 1807
QUERY_SEED = 1409
GEN_VERSION = 5  # bump when any recipe below changes (invalidates the cache)

# ----------------------------------------------------------------------------
# data records
# ----------------------------------------------------------------------------


@dataclass
class Store:
    """Three int32 columns of equal length (SoA), plus the recipe that made them."""
    s: np.ndarray
    p: np.ndarray
    o: np.ndarray
    name: str
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.s.shape[0])

    def triples(self) -> np.ndarray:
        return np.stack([self.s, self.p, self.o], axis=1)


@dataclass
class Pattern:
    """A triple pattern: 0 in s/p/o is "?"; var[j] labels the "?" in slot j (-1: anonymous)."""
    s: int
    p: int
    o: int
    var: tuple = (-1, -1, -1)

    def key(self):
        return (self.s, self.p, self.o)

    def shape(self) -> str:
        return "".join(c if v else "?" for c, v in zip("spo", self.key()))


# ----------------------------------------------------------------------------
# cache
# ----------------------------------------------------------------------------


def _cache_dir() -> str:
    d = os.environ.get("TID_SYNTH_CACHE") or os.path.join(
        os.environ.get("TMPDIR", "/tmp"), "tid_synth_cache")
    os.makedirs(d, exist_ok=True)
    return d


def _cached(tag: str, builder):
    h = hashlib.sha1(f"{tag}|v{GEN_VERSION}".encode()).hexdigest()[:16]
    base = os.path.join(_cache_dir(), h)
    names = ("s", "p", "o")
    if all(os.path.exists(f"{base}.{c}.npy") for c in names):
        return tuple(np.load(f"{base}.{c}.npy") for c in names)
    cols = builder()
    for c, a in zip(names, cols):
        tmp = f"{base}.{c}.{os.getpid()}.tmp.npy"
        np.save(tmp, a)
        os.replace(tmp, f"{base}.{c}.npy")
    return cols


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------


def zipf_cdf(s: float, k: int) -> np.ndarray:
    """CDF of a Zipf(s) law truncated to ranks 1..k (inverse-CDF sampling table)."""
    w = np.arange(1, k + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_ranks(rng: np.random.Generator, n: int, cdf: np.ndarray) -> np.ndarray:
    """n ranks in 1..len(cdf) drawn by inverse CDF."""
    u = rng.random(n)
    r = np.searchsorted(cdf, u, side="right") + 1
    return np.minimum(r, len(cdf)).astype(np.int64)


# packed (s, p, o) key used only to remove duplicate triples:
#   s < 2^26, p < 2^7 (a small predicate value or index), o < 2^31
_S_SHIFT, _P_SHIFT = 38, 31


def _pack(s, pidx, o):
    return (s.astype(np.uint64) << np.uint64(_S_SHIFT)) | \
           (pidx.astype(np.uint64) << np.uint64(_P_SHIFT)) | o.astype(np.uint64)


def _unpack(k):
    s = (k >> np.uint64(_S_SHIFT)).astype(np.int32)
    pidx = ((k >> np.uint64(_P_SHIFT)) & np.uint64(127)).astype(np.int32)
    o = (k & np.uint64((1 << 31) - 1)).astype(np.int32)
    return s, pidx, o


def _sorted_distinct(k: np.ndarray) -> np.ndarray:
    k = np.sort(k)
    if k.shape[0] < 2:
        return k
    keep = np.empty(k.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(k[1:], k[:-1], out=keep[1:])
    return k[keep]


def _unique_topup(rng, n, draw):
    """Draw packed keys until at least n distinct ones exist; keep a seeded n-subset
    in a seeded random order."""
    keys = _sorted_distinct(draw(int(n * 1.08) + 1024))
    while keys.shape[0] < n:
        extra = draw(int((n - keys.shape[0]) * 1.5) + 1024)
        keys = _sorted_distinct(np.concatenate([keys, extra]))
    perm = rng.permutation(keys.shape[0])[:n]
    return keys[perm]


# ----------------------------------------------------------------------------
# tiny workload (1M triples)
# ----------------------------------------------------------------------------

TINY_SUBJECTS = 100_000
TINY_PREDICATES = 64
TINY_OBJECTS = 200_000


def tiny_store(n: int = 1_000_000, seed: int = STORE_SEED) -> Store:
    def build():
        rng = np.random.default_rng(seed)
        cp = zipf_cdf(1.2, TINY_PREDICATES)
        co = zipf_cdf(1.1, TINY_OBJECTS)

        def draw(m):
            s = rng.integers(1, TINY_SUBJECTS + 1, size=m)
            p = zipf_ranks(rng, m, cp)
            o = zipf_ranks(rng, m, co)
            return _pack(s, p, o)

        keys = _unique_topup(rng, n, draw)
        s, p, o = _unpack(keys)
        return (np.ascontiguousarray(s), np.ascontiguousarray(p),
                np.ascontiguousarray(o))

    s, p, o = _cached(f"tiny|{n}|{seed}", build)
    return Store(s, p, o, name=f"tiny-{n}", meta={"seed": seed})


def tiny_queries(store: Store, seed: int = QUERY_SEED, per_shape: int = 4):
    """4 each of (s,?,?), (?,p,?), (?,p,o), (s,p,?), keyed from uniformly drawn
    stored triples (so none is empty)."""
    rng = np.random.default_rng(seed)
    out = []
    for shape in ("s??", "?p?", "?po", "sp?"):
        rows = rng.integers(0, store.n, size=per_shape)
        for r in rows:
            t = (int(store.s[r]), int(store.p[r]), int(store.o[r]))
            key = tuple(t[j] if shape[j] != "?" else 0 for j in range(3))
            var = tuple(-1 if key[j] else j for j in range(3))
            out.append(Pattern(*key, var=var))
    return out


# ----------------------------------------------------------------------------
# university-shaped workload (200M at full size)
# ----------------------------------------------------------------------------

UNI_FULL = 200_000_000
CLASS_FRACTIONS = np.array([.40, .20, .15, .10, .06, .04, .03, .02])
SUBCLASSES = 512         # type objects: each top class has 511 subclasses + itself
PRED_FREQ = np.array([.30, .12, .10, .08, .06, .05, .05, .04, .04, .03,
                      .03, .02, .02, .015, .015, .01, .01, .005, .003, .002])
# per predicate: (kind, domain classes, range classes or literal exponent)
#   kind "type": object is a class ID of the subject's own top class, Zipf(0.5)
#                over its 512 (sub)classes
#   kind "lit":  object is LIT_BASE + uniform[0, 10^k)
#   kind "ent":  object is an entity of the range classes, Zipf(1.1) within a class
PRED_KIND = [
    ("type", range(8), None),
    ("lit", (0, 1), 2),
    ("lit", range(8), 4),
    ("lit", (2, 3), 7),
    ("ent", (0,), (1,)),
    ("lit", (0, 1, 2, 3), 5),
    ("ent", (0, 1), (2,)),
    ("ent", range(8), range(8)),
    ("ent", (1,), (3,)),
    ("lit", (4, 5, 6, 7), 3),
    ("ent", (0,), (0,)),
    ("lit", range(8), 6),
    ("ent", (2, 3), (4, 5)),
    ("ent", (4,), (5,)),
    ("ent", (5, 6), (0,)),
    ("ent", (1, 2), (6, 7)),
    ("ent", (3,), (1, 2)),
    ("ent", (6,), (3,)),
    ("ent", (7,), (0, 1)),
    ("ent", range(8), (7,)),
]


def uni_layout(subjects: int):
    """ID layout of the university store for a given subject count."""
    sizes = np.floor(CLASS_FRACTIONS * subjects).astype(np.int64)
    sizes[0] += subjects - sizes.sum()
    starts = 1 + np.concatenate([[0], np.cumsum(sizes)[:-1]])
    class_base = subjects + 1                       # 8 x 512 class IDs
    pred_base = class_base + 8 * SUBCLASSES         # 20 predicate IDs
    return {"sizes": sizes, "starts": starts, "class_base": class_base,
            "pred_base": pred_base, "pred_ids": pred_base + np.arange(len(PRED_FREQ))}


def uni_subjects(n: int) -> int:
    # 5M subjects at 200M triples (40 triples per subject), scaled with n
    return max(64, n // 40)


def university_store(n: int = UNI_FULL, seed: int = STORE_SEED) -> Store:
    subjects = uni_subjects(n)
    lay = uni_layout(subjects)

    def build():
        rng = np.random.default_rng(seed)
        cdf_sub = zipf_cdf(0.5, SUBCLASSES)
        ccdf = {}

        def class_cdf(c):
            if c not in ccdf:
                ccdf[c] = zipf_cdf(1.1, int(lay["sizes"][c]))
            return ccdf[c]

        sizes, starts = lay["sizes"], lay["starts"]

        def draw_subjects(m, dom):
            dom = np.asarray(list(dom))
            w = sizes[dom] / sizes[dom].sum()
            cls = dom[np.searchsorted(np.cumsum(w), rng.random(m), side="right").clip(0, len(dom) - 1)]
            off = (rng.random(m) * sizes[cls]).astype(np.int64)
            return starts[cls] + off, cls

        def draw(m):
            counts = rng.multinomial(m, PRED_FREQ)
            parts = []
            for j, (kind, dom, rng_or_k) in enumerate(PRED_KIND):
                mj = int(counts[j])
                if mj == 0:
                    continue
                s, cls = draw_subjects(mj, dom)
                if kind == "type":
                    o = lay["class_base"] + cls * SUBCLASSES + (zipf_ranks(rng, mj, cdf_sub) - 1)
                elif kind == "lit":
                    o = LIT_BASE + rng.integers(0, 10 ** rng_or_k, size=mj)
                else:
                    rcls = np.asarray(list(rng_or_k))
                    w = sizes[rcls] / sizes[rcls].sum()
                    pick = rcls[np.searchsorted(np.cumsum(w), rng.random(mj), side="right").clip(0, len(rcls) - 1)]
                    o = np.empty(mj, np.int64)
                    for c in np.unique(pick):
                        sel = pick == c
                        o[sel] = starts[c] + zipf_ranks(rng, int(sel.sum()), class_cdf(int(c))) - 1
                parts.append(_pack(s, np.full(mj, j), o))
            return np.concatenate(parts)

        keys = _unique_topup(rng, n, draw)
        s, pidx, o = _unpack(keys)
        p = lay["pred_ids"][pidx].astype(np.int32)
        return (np.ascontiguousarray(s), np.ascontiguousarray(p),
                np.ascontiguousarray(o))

    s, p, o = _cached(f"uni|{n}|{seed}", build)
    return Store(s, p, o, name=f"university-{n}",
                 meta={"seed": seed, "subjects": subjects, **{k: v for k, v in lay.items()}})


def _tally(a: np.ndarray):
    """Distinct values of a and how often each occurs (sort based)."""
    a = np.sort(a)
    if a.shape[0] == 0:
        return a, np.zeros(0, np.int64)
    start = np.flatnonzero(np.concatenate([[True], a[1:] != a[:-1]]))
    counts = np.diff(np.concatenate([start, [a.shape[0]]]))
    return a[start], counts


def university_queries(store: Store, m: int = 64, seed: int = QUERY_SEED,
                       lo: float = 1e-6, hi: float = 0.3):
    """m single-pattern queries whose result size is as close as the store allows to a
    target selectivity drawn log-uniformly on [lo, hi].  Candidate shapes are
    (?,p,?), (?,p,o), (?,?,o) and (s,?,?); their sizes come from value tallies of
    the store (these choose constants; they are not query answers)."""
    rng = np.random.default_rng(seed)
    n = store.n
    cands = []  # (count, pattern)
    pv, pc = _tally(store.p)
    cands += [(int(c), Pattern(0, int(v), 0, var=(0, -1, 1))) for v, c in zip(pv, pc)]
    po = (store.p.astype(np.int64) << 32) | store.o.astype(np.int64)
    pov, poc = _tally(po)
    ov, oc = _tally(store.o)
    sv, sc = _tally(store.s)
    # keep the candidate lists small: one representative per distinct count bucket
    def reps(vals, counts, mk, per_decade=24):
        keyb = np.floor(np.log10(counts.astype(np.float64)) * per_decade).astype(np.int64)
        _, first = np.unique(keyb, return_index=True)
        return [(int(counts[i]), mk(int(vals[i]))) for i in first]
    cands += reps(pov, poc, lambda x: Pattern(0, x >> 32, x & 0xFFFFFFFF, var=(0, -1, -1)))
    cands += reps(ov, oc, lambda x: Pattern(0, 0, x, var=(0, 1, -1)))
    cands += reps(sv, sc, lambda x: Pattern(x, 0, 0, var=(-1, 0, 1)))
    counts = np.array([c for c, _ in cands], dtype=np.float64)
    targets = np.exp(rng.uniform(np.log(lo), np.log(hi), size=m))
    out = []
    for t in targets:
        i = int(np.argmin(np.abs(np.log(counts) - np.log(t * n))))
        c, pat = cands[i]
        out.append((pat, float(t), c / n))
    return out


# ----------------------------------------------------------------------------
# multi-pattern plans on the university store: star joins, chains, unions, filters
# ----------------------------------------------------------------------------

X, Y, Z, W = 0, 1, 2, 3   # variable ids; extra star variables use 4, 5, ...


def _dom(j):
    return set(PRED_KIND[j][1])


def _rng_classes(j):
    kind, _, r = PRED_KIND[j]
    return set(r) if kind == "ent" else set()


def university_plans(store: Store, seed: int = QUERY_SEED, n_star: int = 16, n_chain: int = 16,
                     n_union: int = 8, n_filter: int = 8):
    """Plans (lists of node dicts, last node = result) of the multi-pattern workload:
    star-shaped joins on one subject (like the paper's five-pattern listing, all SS),
    chains through object->subject joins (like subclass transitivity, OS), unions of
    2-4 subqueries (including overlapping branches), and range FILTERs on encoded
    literals.  Constants are drawn from stored triples' classes and predicates."""
    rng = np.random.default_rng(seed + 7)
    lay = uni_layout(store.meta["subjects"])
    pid = lay["pred_ids"]
    cbase = lay["class_base"]
    ent = [j for j in range(1, len(PRED_KIND)) if PRED_KIND[j][0] == "ent"]
    lit = [j for j in range(1, len(PRED_KIND)) if PRED_KIND[j][0] == "lit"]
    plans = []

    def cls_const(k):
        return int(cbase + k * SUBCLASSES + int(rng.integers(0, 6)))

    def left_deep(nodes, first, rest):
        cur = first
        for r in rest:
            nodes.append({"op": "join", "inputs": [cur, r], "algo": "auto"})
            cur = len(nodes) - 1
        return cur

    for i in range(n_star):
        k = int(rng.choice(8, p=CLASS_FRACTIONS))
        cand = [j for j in range(1, len(PRED_KIND)) if k in _dom(j)]
        npat = int(rng.integers(1, min(4, len(cand)) + 1))
        chosen = [int(x) for x in rng.choice(cand, size=npat, replace=False)]
        nodes = [{"op": "match", "pattern": Pattern(0, int(pid[0]), cls_const(k), var=(X, -1, -1))}]
        for t, j in enumerate(chosen):
            nodes.append({"op": "match", "pattern": Pattern(0, int(pid[j]), 0, var=(X, -1, 4 + t))})
        cur = left_deep(nodes, 0, list(range(1, len(chosen) + 1)))
        if i % 2 == 1:
            nodes.append({"op": "project", "input": cur, "vars": [X, 4]})
        plans.append((f"star{i}", nodes))

    for i in range(n_chain):
        # p_a: range meets the domain of p_b (and p_b's range meets p_c's domain)
        while True:
            a = int(rng.choice(ent))
            nb = [j for j in ent if _rng_classes(a) & _dom(j)]
            if nb:
                break
        b = int(rng.choice(nb))
        k = int(rng.choice(sorted(_dom(a))))
        nodes = [{"op": "match", "pattern": Pattern(0, int(pid[0]), cls_const(k), var=(X, -1, -1))},
                 {"op": "match", "pattern": Pattern(0, int(pid[a]), 0, var=(X, -1, Y))},
                 {"op": "match", "pattern": Pattern(0, int(pid[b]), 0, var=(Y, -1, Z))}]
        rest = [1, 2]
        nc = [j for j in ent if _rng_classes(b) & _dom(j)]
        if i % 3 == 2 and nc:
            c = int(rng.choice(nc))
            nodes.append({"op": "match", "pattern": Pattern(0, int(pid[c]), 0, var=(Z, -1, W))})
            rest.append(3)
        cur = left_deep(nodes, 0, rest)
        nodes.append({"op": "project", "input": cur, "vars": [X, Z]})
        plans.append((f"chain{i}", nodes))

    for i in range(n_union):
        r = int(rng.integers(0, store.n))
        s0 = int(store.s[r])
        nb = 2 + i % 3
        nodes = []
        if i % 4 == 3:
            # overlapping branches: (s ?p ?o) UNION (?s p ?o), a triple may answer both
            p0 = int(store.p[r])
            nodes.append({"op": "match", "pattern": Pattern(s0, 0, 0, var=(-1, X, Y))})
            nodes.append({"op": "match", "pattern": Pattern(0, p0, int(store.o[r]), var=(Z, -1, -1))})
            nodes.append({"op": "union", "inputs": [0, 1]})
        else:
            # same subject, different predicates: (s p_j ?v), mostly predicates s has
            own = np.unique(store.p[store.s == s0])
            js = [int(x) for x in rng.choice(own, size=min(nb - 1, len(own)), replace=False)]
            js.append(int(pid[int(rng.integers(0, len(pid)))]))
            for pj in js:
                nodes.append({"op": "match", "pattern": Pattern(s0, pj, 0, var=(-1, -1, Y))})
            nb = len(js)
            nodes.append({"op": "union", "inputs": list(range(nb))})
        plans.append((f"union{i}", nodes))

    for i in range(n_filter):
        j = int(rng.choice(lit))
        kexp = PRED_KIND[j][2]
        lo = int(rng.integers(0, 10 ** kexp // 2))
        hi = lo + int(10 ** kexp * rng.uniform(0.001, 0.2))
        k = int(rng.choice(sorted(_dom(j))))
        nodes = [{"op": "match", "pattern": Pattern(0, int(pid[j]), 0, var=(X, -1, Y))},
                 {"op": "filter", "input": 0, "var": Y, "cmp": "range", "a": LIT_BASE + lo, "b": LIT_BASE + hi}]
        if i % 2 == 0:
            nodes.append({"op": "match", "pattern": Pattern(0, int(pid[0]), cls_const(k), var=(X, -1, -1))})
            nodes.append({"op": "join", "inputs": [1, 2], "algo": "auto"})
        plans.append((f"filter{i}", nodes))
    return plans


# ----------------------------------------------------------------------------
# large stores drawn on a device (batched and served workloads: 500M, 1B)
# ----------------------------------------------------------------------------
#
# The same university recipe as university_store, drawn with torch on a device
# (seconds at 500M, where the host recipe takes minutes).  The values differ from
# university_store's (another random stream); the recipe, the ID layout and the
# set property are the same.  Inputs only: no matching, joining or compaction.


def university_store_torch(n: int, seed: int = STORE_SEED, device="cuda"):
    """(s, p, o) int32 tensors on `device`: n distinct triples of the university
    recipe in a seeded random order."""
    import torch
    dev = torch.device(device)
    subjects = uni_subjects(n)
    lay = uni_layout(subjects)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    hrng = np.random.default_rng(seed)
    sizes = torch.as_tensor(lay["sizes"], dtype=torch.int64, device=dev)
    starts = torch.as_tensor(lay["starts"], dtype=torch.int64, device=dev)
    cdf_sub = torch.as_tensor(zipf_cdf(0.5, SUBCLASSES), device=dev)
    ccdf = {}

    def zipf(m, cdf):
        u = torch.rand(m, generator=g, device=dev, dtype=torch.float64)
        return torch.searchsorted(cdf, u, right=True).clamp_(max=cdf.shape[0] - 1) + 1

    def pick(m, classes):
        cls = torch.as_tensor(sorted(classes), dtype=torch.int64, device=dev)
        w = torch.cumsum(sizes[cls].double(), 0)
        u = torch.rand(m, generator=g, device=dev, dtype=torch.float64) * w[-1]
        return cls[torch.searchsorted(w, u, right=True).clamp_(max=cls.shape[0] - 1)]

    def draw(m):
        counts = hrng.multinomial(m, PRED_FREQ)
        parts = []
        for j, (kind, dom, r) in enumerate(PRED_KIND):
            mj = int(counts[j])
            if mj == 0:
                continue
            cls = pick(mj, dom)
            off = (torch.rand(mj, generator=g, device=dev, dtype=torch.float64) * sizes[cls]).long()
            s = starts[cls] + off
            if kind == "type":
                o = lay["class_base"] + cls * SUBCLASSES + (zipf(mj, cdf_sub) - 1)
            elif kind == "lit":
                o = LIT_BASE + torch.randint(0, 10 ** r, (mj,), generator=g, device=dev)
            else:
                rc = pick(mj, r)
                o = torch.empty(mj, dtype=torch.int64, device=dev)
                for c in sorted(set(r)):
                    sel = rc == c
                    k = int(sel.sum())
                    if k:
                        if c not in ccdf:
                            ccdf[c] = torch.as_tensor(zipf_cdf(1.1, int(lay["sizes"][c])), device=dev)
                        o[sel] = int(lay["starts"][c]) + zipf(k, ccdf[c]) - 1
            parts.append((s << _S_SHIFT) | (j << _P_SHIFT) | o)
        return torch.cat(parts)

    keys = torch.unique(draw(int(n * 1.08) + 1024))
    while keys.shape[0] < n:
        keys = torch.unique(torch.cat([keys, draw(int((n - keys.shape[0]) * 1.5) + 1024)]))
    keys = keys[torch.randperm(keys.shape[0], generator=g, device=dev)[:n]]
    s = ((keys >> _S_SHIFT) & ((1 << 26) - 1)).int()
    pidx = (keys >> _P_SHIFT) & 127
    o = (keys & ((1 << 31) - 1)).int()
    del keys
    p = torch.as_tensor(lay["pred_ids"], dtype=torch.int64, device=dev)[pidx].int()
    return s.contiguous(), p.contiguous(), o.contiguous()


# (mask, shape name, var labels) of the single-pattern shapes a batch draws from
BATCH_SHAPES = [(2, "?p?", (0, -1, 1)), (6, "?po", (0, -1, -1)), (4, "??o", (0, 1, -1)),
                (1, "s??", (-1, 0, 1)), (3, "sp?", (-1, -1, 0)), (5, "s?o", (-1, 0, -1)),
                (7, "spo", (-1, -1, -1))]


def batch_queries(s, p, o, m: int = 4096, seed: int = QUERY_SEED, lo: float = 1.0, hi: float = 1e7,
                  window: float = 1.5):
    """m single-pattern queries whose result sizes are log-uniform on [lo, hi] as far as
    the store allows.  For each target size t a shape is drawn among those having
    patterns whose size lies within a factor `window` of t, then one such pattern at
    random (so a batch holds many distinct keys of every size); if no shape has one,
    the pattern whose size is closest to t.  Sizes come from value tallies of the
    store's columns (torch tensors, any device); they choose constants only.
    Returns a list of (Pattern, target size, tally size)."""
    import torch
    rng = np.random.default_rng(seed + 4096)
    s64, p64, o64 = s.long(), p.long(), o.long()
    cols = {1: s64, 2: p64, 4: o64}
    targets = np.exp(rng.uniform(np.log(lo), np.log(hi), size=m))
    tt = torch.as_tensor(targets, device=s.device)
    shapes = []
    for mask, name, var in BATCH_SHAPES:
        bound = [b for b in (1, 2, 4) if mask & b]
        if len(bound) == 3:  # (s, p, o): every stored triple is a size-1 pattern
            vals, cnt = None, None
        else:
            key = cols[bound[0]] if len(bound) == 1 else cols[bound[0]] * (1 << 32) + cols[bound[1]]
            vals, cnt = torch.unique(key, return_counts=True)
            del key
            order = torch.argsort(cnt)
            vals, cnt = vals[order], cnt[order]
        shapes.append((mask, var, bound, vals, cnt))
    n = s.shape[0]
    lo_t, hi_t = (tt / window).ceil(), (tt * window).floor()
    choice = []
    for mask, var, bound, vals, cnt in shapes:
        if cnt is None:
            a = torch.zeros(m, dtype=torch.int64, device=s.device)
            b = torch.where((lo_t <= 1) & (hi_t >= 1), torch.full_like(a, n), a)
        else:
            a = torch.searchsorted(cnt, lo_t.long())
            b = torch.searchsorted(cnt, hi_t.long(), right=True)
        choice.append((a.cpu().numpy(), b.cpu().numpy()))
    out = []
    for i, t in enumerate(targets):
        ok = [k for k in range(len(shapes)) if choice[k][1][i] > choice[k][0][i]]
        if ok:
            k = int(rng.choice(ok))
            j = int(rng.integers(choice[k][0][i], choice[k][1][i]))
        else:  # closest size over all shapes
            best = None
            for k2, (_, _, _, vals, cnt) in enumerate(shapes):
                if cnt is None:
                    continue
                q = int(torch.searchsorted(cnt, torch.as_tensor([int(t)], device=cnt.device)).clamp(max=cnt.shape[0] - 1))
                for jj in (max(0, q - 1), q):
                    d = abs(np.log(float(cnt[jj])) - np.log(t))
                    if best is None or d < best[0]:
                        best = (d, k2, jj)
            _, k, j = best
        mask, var, bound, vals, cnt = shapes[k]
        if vals is None:
            r = j
            key = {1: int(s[r]), 2: int(p[r]), 4: int(o[r])}
            size = 1
        else:
            v = int(vals[j])
            if len(bound) == 1:
                key = {bound[0]: v}
            else:
                key = {bound[0]: v >> 32, bound[1]: v & 0xFFFFFFFF}
            size = int(cnt[j])
        pat = Pattern(key.get(1, 0), key.get(2, 0), key.get(4, 0), var=var)
        out.append((pat, float(t), size))
    return out


# ----------------------------------------------------------------------------
# a served request stream: Poisson arrivals of three query classes
# ----------------------------------------------------------------------------

# index lookups, two-pattern star joins, unions / filters, wide scans, typed star joins
SERVE_MIX = (0.68, 0.14, 0.14, 0.02, 0.02)


def serving_requests(s, p, o, m: int = 4000, seed: int = QUERY_SEED, mix=SERVE_MIX, hi_index: float = 1e5,
                     rate: float = 20000.0):
    """m requests over a university store held as torch columns, with Poisson
    arrival offsets (seconds, mean rate `rate`).  Returns (kinds, payloads,
    arrivals): kind "index" carries a Pattern (the answer is its index list); kind
    "plan" carries a plan (list of node dicts).  The classes, drawn with
    probabilities `mix` (a shorter mix leaves the later classes out):
      0 index lookups: result sizes log-uniform on [1, hi_index] (as batch_queries);
      1 star: (?X p1 o1) JOIN (?X p2 o2), two triples of one random subject whose
        predicates are entity-valued or fine-grained literals (both selective);
      2 union: (s p_j ?Y) for 2-4 predicates of one random subject, UNION; or
        filter: (s ?P ?V) of one random subject, FILTER ?V in a literal range;
      3 wide scans (the large-scan class): one pattern whose result size is
        log-uniform on [1e5, 0.3 n];
      4 typed star joins (the multi-pattern class): (?X type C) JOIN (?X p ?Y),
        C one of the four most frequent subclasses of a top class in p's domain
        and p entity-valued with frequency <= 0.02, so the intermediates hold
        0.1-20M rows at 1B triples.
    Inputs only: subjects and their triples are looked up by sorting the subject
    column (no query evaluation)."""
    import torch
    rng = np.random.default_rng(seed + 20000)
    mix = np.asarray(mix, np.float64)
    kinds = rng.choice(len(mix), size=m, p=mix / mix.sum())
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=m))
    n = int(s.shape[0])
    lay = uni_layout(uni_subjects(n))
    pred_base = int(lay["pred_base"])
    selective = set()
    for j, (kind, _, r) in enumerate(PRED_KIND):
        if kind == "ent" or (kind == "lit" and r >= 5):
            selective.add(pred_base + j)
    n_index = int((kinds == 0).sum())
    idx_q = iter(batch_queries(s, p, o, m=n_index, seed=seed + 1, lo=1.0, hi=hi_index) if n_index else [])
    n_wide = int((kinds == 3).sum())
    wide_q = iter(batch_queries(s, p, o, m=n_wide, seed=seed + 2, lo=1e5, hi=max(2e5, 0.3 * n)) if n_wide else [])
    heavy_preds = [(j, dom) for j, (kind, dom, _) in enumerate(PRED_KIND) if kind == "ent" and PRED_FREQ[j] <= 0.02]
    s_sorted, order = torch.sort(s)

    def triples_of(s0):
        a = int(torch.searchsorted(s_sorted, torch.tensor([s0], dtype=s_sorted.dtype, device=s.device)))
        b = int(torch.searchsorted(s_sorted, torch.tensor([s0], dtype=s_sorted.dtype, device=s.device), right=True))
        rows = order[a:b]
        return p[rows].cpu().numpy(), o[rows].cpu().numpy()

    def random_subject():
        return int(s[int(rng.integers(0, n))])

    payloads = []
    for kd in kinds:
        if kd == 0:
            payloads.append(next(idx_q)[0])
            continue
        if kd == 3:
            payloads.append(next(wide_q)[0])
            continue
        if kd == 4:
            j, dom = heavy_preds[int(rng.integers(0, len(heavy_preds)))]
            cls = int(rng.choice(np.asarray(list(dom))))
            c_id = int(lay["class_base"]) + cls * SUBCLASSES + int(rng.integers(0, 4))
            payloads.append([{"op": "match", "pattern": Pattern(0, pred_base, c_id, var=(X, -1, -1))},
                             {"op": "match", "pattern": Pattern(0, pred_base + j, 0, var=(X, -1, Y))},
                             {"op": "join", "inputs": [0, 1], "algo": "auto"}])
            continue
        while True:
            s0 = random_subject()
            ps, os_ = triples_of(s0)
            if kd == 1:
                cand = [i for i in range(len(ps)) if int(ps[i]) in selective]
                if len(cand) < 2:
                    continue
                i1, i2 = (int(x) for x in rng.choice(cand, size=2, replace=False))
                plan = [{"op": "match", "pattern": Pattern(0, int(ps[i1]), int(os_[i1]), var=(X, -1, -1))},
                        {"op": "match", "pattern": Pattern(0, int(ps[i2]), int(os_[i2]), var=(X, -1, -1))},
                        {"op": "join", "inputs": [0, 1], "algo": "auto"}]
            elif rng.random() < 0.5:
                own = np.unique(ps)
                if len(own) < 2:
                    continue
                k = int(rng.integers(2, min(4, len(own)) + 1))
                plan = [{"op": "match", "pattern": Pattern(s0, int(pj), 0, var=(-1, -1, Y))}
                        for pj in rng.choice(own, size=k, replace=False)]
                plan.append({"op": "union", "inputs": list(range(k))})
            else:
                lit = os_[os_ >= LIT_BASE]
                if len(lit) == 0:
                    continue
                v = int(rng.choice(lit)) - LIT_BASE
                lo_, hi_ = max(0, v - int(rng.integers(0, 1000))), v + int(rng.integers(0, 1000))
                plan = [{"op": "match", "pattern": Pattern(s0, 0, 0, var=(-1, Y, Z))},
                        {"op": "filter", "input": 0, "var": Z, "cmp": "range",
                         "a": LIT_BASE + lo_, "b": LIT_BASE + hi_}]
            payloads.append(plan)
            break
    del s_sorted, order
    return ["index" if k in (0, 3) else "plan" for k in kinds], payloads, arrivals


# ----------------------------------------------------------------------------
# an RDFS schema for the university store (entailment workload)
# ----------------------------------------------------------------------------

# (sub-property, super-property) by predicate index: two chains of length two
# (10 -> 4 -> 7 -> 19 and 6 -> 7) and two single links
SUBPROPS = [(4, 7), (6, 7), (7, 19), (10, 4), (13, 12), (16, 15)]


def rdfs_vocab(subjects: int) -> dict:
    """IDs of rdf:type (the store's type predicate) and of the four schema
    predicates, placed after the store's 20 predicate IDs."""
    lay = uni_layout(subjects)
    base = int(lay["pred_base"]) + len(PRED_FREQ)
    return {"type": int(lay["pred_ids"][0]), "domain": base, "range": base + 1, "subprop": base + 2,
            "subclass": base + 3}


def rdfs_schema(subjects: int):
    """Schema triples (s, p, o int32 arrays) of the university store: each top class's
    512 (sub)class IDs form a binary subClassOf tree under the top class, top
    classes 1..7 are subclasses of top class 0; every predicate has rdfs:domain its
    domain classes' top classes, entity predicates rdfs:range their range classes'
    top classes; SUBPROPS are subPropertyOf links."""
    lay = uni_layout(subjects)
    v = rdfs_vocab(subjects)
    pid = [int(x) for x in lay["pred_ids"]]
    cb = int(lay["class_base"])

    def cls(k, j):
        return cb + k * SUBCLASSES + j

    t = []
    for k in range(len(CLASS_FRACTIONS)):
        for j in range(1, SUBCLASSES):
            t.append((cls(k, j), v["subclass"], cls(k, (j - 1) // 2)))
        if k:
            t.append((cls(k, 0), v["subclass"], cls(0, 0)))
    for j in range(1, len(PRED_KIND)):
        kind, dom, rng_ = PRED_KIND[j]
        for c in sorted(set(dom)):
            t.append((pid[j], v["domain"], cls(c, 0)))
        if kind == "ent":
            for c in sorted(set(rng_)):
                t.append((pid[j], v["range"], cls(c, 0)))
    for a, b in SUBPROPS:
        t.append((pid[a], v["subprop"], pid[b]))
    a = np.array(sorted(set(t)), np.int32)
    return a[:, 0].copy(), a[:, 1].copy(), a[:, 2].copy()


def with_schema(store: Store) -> Store:
    """The store followed by its schema triples (still a set: the schema uses
    predicates the data does not)."""
    ss, sp, so = rdfs_schema(store.meta["subjects"])
    return Store(np.concatenate([store.s, ss]), np.concatenate([store.p, sp]), np.concatenate([store.o, so]),
                 name=store.name + "+rdfs", meta=dict(store.meta, schema_triples=int(ss.shape[0])))
