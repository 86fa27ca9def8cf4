// Single-pass row compaction over tuple sets, and a device-wide exclusive scan.
//
// One kernel template serves the operators that keep a subset of rows in
// their original order and write k output columns:
//   * bind     -- from triple indices, the terms at a pattern's variable slots,
//                 dropping rows whose repeated variable disagrees; the FILTER
//                 predicates of the subquery are applied in the same pass
//                 (Section 4.3: the filter is applied while the matched triples
//                 are extracted into the subquery's vector);
//   * filter   -- a predicate on one column of a set;
//   * unique   -- after a sort, a row is kept when it differs from its
//                 predecessor in sorted order (DISTINCT, Section 4.3), on
//                 column rows or on packed row keys;
//   * semijoin -- the entailment's keyed store pass (Section 5): a store triple
//                 is kept when its term at the join position is one of the
//                 first search's distinct terms (a hash probe).
// A CTA owns 2048 consecutive rows (256 threads x 8, striped so each warp
// instruction touches 32 consecutive rows); ranks come from ballots, the
// tile offset from the decoupled look-back (lookback.cuh).

#include <algorithm>

#include "lookback.cuh"
#include "ops.cuh"

namespace tid {

namespace {

constexpr int CP_THREADS = 256;
constexpr int CP_WARPS = CP_THREADS / 32;
constexpr int CP_ITEMS = 8;
constexpr int CP_TILE = CP_THREADS * CP_ITEMS;

__device__ __forceinline__ bool pred_ok(const Pred &p, int32_t x) {
    if (x == 0) return false;  // unbound never passes
    switch (p.op) {
        case TID_CMP_EQ: return x == p.a;
        case TID_CMP_NE: return x != p.a;
        case TID_CMP_LT: return x < p.a;
        case TID_CMP_LE: return x <= p.a;
        case TID_CMP_GT: return x > p.a;
        case TID_CMP_GE: return x >= p.a;
        case TID_CMP_RANGE: return p.a <= x && x <= p.b;
        default: return false;
    }
}

// ---- row sources -----------------------------------------------------------

// A row source says, for a row r < n, whether it is kept (keep: reads only
// what the test needs) and gives its k output values (values: v[0..k)).
// Column loops run to TID_MAX_COLS with a guard so v[] stays in registers.

__device__ __forceinline__ bool preds_ok(const Pred *preds, int n_preds, const int32_t *v) {
    bool ok = true;
#pragma unroll
    for (int q = 0; q < MAX_PREDS; ++q) {
        if (q < n_preds) {
            int32_t x = v[0];
#pragma unroll
            for (int c = 1; c < TID_MAX_COLS; ++c)
                if (preds[q].col == c) x = v[c];
            ok = ok && pred_ok(preds[q], x);
        }
    }
    return ok;
}

struct BindRow {  // triple index -> variable values
    const int32_t *S, *P, *O;
    const int32_t *idx;
    int k;
    int need;                   // slots (bit 0 s, 1 p, 2 o) that carry a variable
    int8_t src[TID_MAX_COLS];   // slot (0,1,2) giving output column c
    int8_t eq_a[3], eq_b[3];    // pairs of slots that must be equal
    int n_eq;
    Pred preds[MAX_PREDS];
    int n_preds;
    __device__ __forceinline__ void slots(int64_t r, int32_t &t0, int32_t &t1, int32_t &t2) const {
        const int64_t t = idx[r];
        // only the variable slots are read: a bound slot holds the key itself
        t0 = (need & 1) ? S[t] : 0;
        t1 = (need & 2) ? P[t] : 0;
        t2 = (need & 4) ? O[t] : 0;
    }
    __device__ __forceinline__ void out_of(int32_t t0, int32_t t1, int32_t t2, int32_t *v) const {
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) v[c] = src[c] == 0 ? t0 : (src[c] == 1 ? t1 : t2);
    }
    __device__ __forceinline__ bool keep(int64_t r) const {
        if (n_eq == 0 && n_preds == 0) return true;
        int32_t t0, t1, t2, v[TID_MAX_COLS];
        slots(r, t0, t1, t2);
        bool ok = true;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            if (e < n_eq) {
                const int32_t a = eq_a[e] == 0 ? t0 : (eq_a[e] == 1 ? t1 : t2);
                const int32_t b = eq_b[e] == 0 ? t0 : (eq_b[e] == 1 ? t1 : t2);
                ok = ok && a == b;
            }
        }
        out_of(t0, t1, t2, v);
        return ok && preds_ok(preds, n_preds, v);
    }
    __device__ __forceinline__ void values(int64_t r, int32_t *v) const {
        int32_t t0, t1, t2;
        slots(r, t0, t1, t2);
        out_of(t0, t1, t2, v);
    }
};

struct FilterRow {
    const int32_t *col[TID_MAX_COLS];
    int k;
    Pred preds[MAX_PREDS];
    int n_preds;
    __device__ __forceinline__ bool keep(int64_t r) const {  // the predicates' columns only
        bool ok = true;
#pragma unroll
        for (int q = 0; q < MAX_PREDS; ++q) {
            if (q < n_preds) {
                const int32_t *cp = col[0];  // selected with constant indices (no local copy of col[])
#pragma unroll
                for (int c = 1; c < TID_MAX_COLS; ++c)
                    if (preds[q].col == c) cp = col[c];
                ok = ok && pred_ok(preds[q], cp[r]);
            }
        }
        return ok;
    }
    __device__ __forceinline__ void values(int64_t r, int32_t *v) const {
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) v[c] = col[c][r];
    }
};

struct UniqueRow {  // rows in perm order; keep the first of each run of equal rows
    const int32_t *col[TID_MAX_COLS];
    const int32_t *perm;  // may be null (rows already in order)
    int k;
    __device__ __forceinline__ bool keep(int64_t r) const {
        if (r == 0) return true;
        const int64_t a = perm ? perm[r] : r;
        const int64_t b = perm ? perm[r - 1] : r - 1;
        bool same = true;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) same = same && col[c][b] == col[c][a];
        return !same;
    }
    __device__ __forceinline__ void values(int64_t r, int32_t *v) const {
        const int64_t a = perm ? perm[r] : r;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) v[c] = col[c][a];
    }
};

struct SemiJoinRow {  // store triple r, kept when a slot holds a fixed term and another slot's
                      // term is in a key set (open-addressing table of keys, 0 = empty)
    const int32_t *S, *P, *O;
    int need;                   // slots read (bit 0 s, 1 p, 2 o)
    int fixed_slot;             // -1: none
    int32_t fixed_val;
    int key_slot;
    const int32_t *table;
    int tbits;                  // log2 of the table size
    int k;
    int8_t src[TID_MAX_COLS];   // slot giving output column c
    __device__ __forceinline__ const int32_t *column(int slot) const { return slot == 0 ? S : (slot == 1 ? P : O); }
    // the fixed column first, the key column and a probe only for rows that pass
    __device__ __forceinline__ bool keep(int64_t r) const {
        return keep_given(r, first_column()[r]);
    }
    // the column tested first: the fixed one, else the key column
    __device__ __forceinline__ const int32_t *first_column() const {
        return column(fixed_slot >= 0 ? fixed_slot : key_slot);
    }
    // keep(r), given v = first_column()[r]
    __device__ __forceinline__ bool keep_given(int64_t r, int32_t v) const {
        if (fixed_slot >= 0 && v != fixed_val) return false;
        const int32_t key = fixed_slot >= 0 ? column(key_slot)[r] : v;
        if (key == 0) return false;
        const uint32_t tmask = (1u << tbits) - 1u;
        uint32_t h = ((uint32_t)key * 0x9E3779B1u) >> (32 - tbits);  // top bits: all of the key counts
        for (uint32_t probe = 0; probe <= tmask; ++probe) {  // the table is at most half full
            const int32_t e = __ldg(table + h);
            if (e == key) return true;
            if (e == 0) return false;
            h = (h + 1) & tmask;
        }
        return false;
    }
    __device__ __forceinline__ void values(int64_t r, int32_t *v) const {
        const int32_t t0 = (need & 1) ? S[r] : 0;
        const int32_t t1 = (need & 2) ? P[r] : 0;
        const int32_t t2 = (need & 4) ? O[r] : 0;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) v[c] = src[c] == 0 ? t0 : (src[c] == 1 ? t1 : t2);
    }
};

template <typename K>
struct PackedUniqueRow {  // sorted packed keys; keep the first of each run of equal keys
    const K *keys;
    PackSpec ps;
    int k;
    __device__ __forceinline__ bool keep(int64_t r) const { return r == 0 || keys[r - 1] != keys[r]; }
    __device__ __forceinline__ void values(int64_t r, int32_t *v) const {
        const K key = keys[r];
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c < k) {
                const uint32_t f = ps.mask[c] ? (uint32_t)((key >> ps.shift[c]) & ps.mask[c]) : 0u;
                v[c] = (int32_t)((f + ps.min[c]) ^ 0x80000000u);
            }
        }
    }
};

// bounds (sort order) of the values a thread wrote, merged per warp into mm
__device__ __forceinline__ void merge_bounds(uint32_t *mm, int k_out, const uint32_t *lo, const uint32_t *hi) {
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        if (c < k_out) {
            uint32_t a = lo[c], b = hi[c];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                a = min(a, __shfl_xor_sync(0xffffffffu, a, d));
                b = max(b, __shfl_xor_sync(0xffffffffu, b, d));
            }
            // the bounds only tighten, so a warp that cannot improve the
            // current one (read from L2; a stale read only costs an atomic)
            // skips its atomic: many warps otherwise queue on one address
            if (lane == 0 && a <= b) {
                if (a < __ldcg(mm + c)) atomicMin(mm + c, a);
                if (b > __ldcg(mm + TID_MAX_COLS + c)) atomicMax(mm + TID_MAX_COLS + c, b);
            }
        }
    }
}

// ---- single-pass compaction (small inputs) ----------------------------------------

// The tile's kept rows are staged in shared memory at their place in the tile
// (the block's own scan gives it) while warp 0 looks back for the tile's
// offset, so the value reads overlap that wait; the tile is then written with
// coalesced stores.  Dynamic shared memory: k_out x CP_TILE int32.
template <class Row>
__global__ void __launch_bounds__(CP_THREADS)
k_compact(Row row, int64_t n, int k_out, OutCols out, int64_t cap, int64_t *__restrict__ d_rows,
          int64_t *__restrict__ h_rows, Lookback lb, uint32_t *__restrict__ mm) {
    extern __shared__ int32_t s_vals[];  // column c of staged row i at s_vals[c * CP_TILE + i]
    __shared__ unsigned s_tile, s_total;
    __shared__ unsigned s_off[CP_ITEMS * CP_WARPS];
    __shared__ long long s_prefix;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = lb_ticket(lb);
    __syncthreads();
    const unsigned tile = s_tile;
    if (tile >= lb.num_tiles) return;
    const int64_t base = (int64_t)tile * CP_TILE;
    const unsigned lt = (1u << lane) - 1u;

    unsigned keep = 0, wpre[CP_ITEMS];
    bool kp[CP_ITEMS];
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) {  // all tests first: their loads are in flight together
        const int64_t r = base + j * CP_THREADS + threadIdx.x;
        kp[j] = row.keep(r < n ? r : n - 1) && r < n;  // rows past n test row n - 1 and are dropped
    }
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) {
        keep |= (unsigned)kp[j] << j;
        const unsigned b = __ballot_sync(0xffffffffu, kp[j]);
        wpre[j] = __popc(b & lt);
        if (lane == 0) s_off[j * CP_WARPS + warp] = __popc(b);
    }
    __syncthreads();
    if (warp == 0) {  // 64 (item, warp) counts in order; each lane scans two consecutive entries
        const unsigned a0 = s_off[2 * lane], a1 = s_off[2 * lane + 1];
        unsigned x = a0 + a1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += y;
        }
        const unsigned ex = x - a0 - a1;
        s_off[2 * lane] = ex;
        s_off[2 * lane + 1] = ex + a0;
        if (lane == 31) s_total = x;
    }
    __syncthreads();
    const unsigned total = s_total;
    auto stage = [&]() {  // this thread's kept rows to their place in the tile
#pragma unroll
        for (int j = 0; j < CP_ITEMS; ++j) {
            if (!((keep >> j) & 1u)) continue;
            int32_t v[TID_MAX_COLS];
            row.values(base + j * CP_THREADS + threadIdx.x, v);
            const unsigned at = s_off[j * CP_WARPS + warp] + wpre[j];
#pragma unroll
            for (int c = 0; c < TID_MAX_COLS; ++c)
                if (c < k_out) s_vals[c * CP_TILE + at] = v[c];
        }
    };
    if (warp == 0) {
        const long long excl = lb_exclusive_prefix(lb, tile, total);
        if (lane == 0) {
            s_prefix = excl;
            if (tile == lb.num_tiles - 1 && excl >= 0) {
                *d_rows = excl + total;
                *h_rows = excl + total;
            }
        }
    }
    stage();  // warps 1.. stage while warp 0 waits for the tile's offset
    __syncthreads();
    const long long prefix = s_prefix;
    if (prefix < 0) return;
    uint32_t lo[TID_MAX_COLS], hi[TID_MAX_COLS];
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        lo[c] = 0xFFFFFFFFu;
        hi[c] = 0u;
    }
    for (unsigned i = threadIdx.x; i < total; i += CP_THREADS) {  // coalesced: row prefix + i
        const long long pos = prefix + i;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c < k_out) {
                const int32_t v = s_vals[c * CP_TILE + i];
                if (pos < cap) out.col[c][pos] = v;
                const uint32_t u = (uint32_t)v ^ 0x80000000u;
                lo[c] = min(lo[c], u);
                hi[c] = max(hi[c], u);
            }
        }
    }
    if (mm) merge_bounds(mm, k_out, lo, hi);  // column bounds of the kept rows
}

// ---- two-kernel compaction (dense keeps over long inputs) -------------------------
//
// k_tile_counts: every CTA tests its 2048-row tile and writes the tile's count;
// the counts are scanned (k_scan_u32); k_tile_write tests the tile again, ranks
// its kept rows (ballots and a block scan), stages their values in shared memory
// and writes them at the tile's offset with coalesced stores.  No CTA waits for
// another; the test columns are read twice.

template <class Row>
__global__ void __launch_bounds__(CP_THREADS) k_tile_counts(Row row, int64_t n, uint32_t *__restrict__ counts) {
    __shared__ unsigned s_w[CP_WARPS];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * CP_TILE;
    bool kp[CP_ITEMS];
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) {
        const int64_t r = base + j * CP_THREADS + threadIdx.x;
        kp[j] = row.keep(r < n ? r : n - 1) && r < n;
    }
    unsigned c = 0;
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) c += __popc(__ballot_sync(0xffffffffu, kp[j]));
    if (lane == 0) s_w[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < CP_WARPS; ++w) t += s_w[w];
        counts[blockIdx.x] = t;
    }
}

template <class Row>
__global__ void __launch_bounds__(CP_THREADS)
k_tile_write(Row row, int64_t n, int k_out, OutCols out, int64_t cap, const uint32_t *__restrict__ offs,
             const uint32_t *__restrict__ counts, unsigned tiles, int64_t *__restrict__ d_rows,
             int64_t *__restrict__ h_rows, uint32_t *__restrict__ mm) {
    extern __shared__ int32_t s_vals[];  // column c of staged row i at s_vals[c * CP_TILE + i]
    __shared__ unsigned s_off[CP_ITEMS * CP_WARPS];
    __shared__ unsigned s_total;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * CP_TILE;
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // the result's row count
        const int64_t total = (int64_t)offs[tiles - 1] + counts[tiles - 1];
        *d_rows = total;
        *h_rows = total;
    }
    bool kp[CP_ITEMS];
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) {
        const int64_t r = base + j * CP_THREADS + threadIdx.x;
        kp[j] = row.keep(r < n ? r : n - 1) && r < n;
    }
    unsigned keep = 0, wpre[CP_ITEMS];
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) {
        keep |= (unsigned)kp[j] << j;
        const unsigned b = __ballot_sync(0xffffffffu, kp[j]);
        wpre[j] = __popc(b & lt);
        if (lane == 0) s_off[j * CP_WARPS + warp] = __popc(b);
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned a0 = s_off[2 * lane], a1 = s_off[2 * lane + 1];
        unsigned x = a0 + a1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += y;
        }
        const unsigned ex = x - a0 - a1;
        s_off[2 * lane] = ex;
        s_off[2 * lane + 1] = ex + a0;
        if (lane == 31) s_total = x;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) {
        if (!((keep >> j) & 1u)) continue;
        int32_t v[TID_MAX_COLS];
        row.values(base + j * CP_THREADS + threadIdx.x, v);
        const unsigned at = s_off[j * CP_WARPS + warp] + wpre[j];
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k_out) s_vals[c * CP_TILE + at] = v[c];
    }
    __syncthreads();
    const unsigned total = s_total;
    const long long o0 = offs[blockIdx.x];
    uint32_t lo[TID_MAX_COLS], hi[TID_MAX_COLS];
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        lo[c] = 0xFFFFFFFFu;
        hi[c] = 0u;
    }
    for (unsigned i = threadIdx.x; i < total; i += CP_THREADS) {
        const long long pos = o0 + i;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c < k_out) {
                const int32_t v = s_vals[c * CP_TILE + i];
                if (pos < cap) out.col[c][pos] = v;
                const uint32_t u = (uint32_t)v ^ 0x80000000u;
                lo[c] = min(lo[c], u);
                hi[c] = max(hi[c], u);
            }
        }
    }
    if (mm) merge_bounds(mm, k_out, lo, hi);
}

// ---- bitmap compaction (large inputs): K1's structure for rows --------------------
//
// One cooperative launch.  Phase A: warps draw runs of BC_DRAW steps of 1024
// rows from one counter; for step j a warp tests rows 1024 j + 32 w + lane
// (w = 0..31, BC_INFLIGHT tests in flight per lane), keeps the 32 ballots as the
// step's keep words and its count, and adds the count to the total of the CTA
// whose fixed range of steps holds it.  Bounded grid barrier.  Phase C: CTA
// c's offset is the sum of the earlier CTAs' totals; it block-scans its steps'
// counts and a warp expands a step: the kept rows' positions in the step go
// to a shared-memory stage (popc, warp scan, set bits), then the warp reads
// the kept rows' values in row order and writes them with coalesced stores.
// A tile never waits for a slower predecessor: the only wait is the barrier.

constexpr int BC_THREADS = 256;
constexpr int BC_WARPS = BC_THREADS / 32;
constexpr int BC_INFLIGHT = 16;    // rows a lane tests at once (their loads in flight together)

// kp[u] = row.keep(row base + 32 u) for u < BC_INFLIGHT (false past n)
template <class Row>
__device__ __forceinline__ void keep_batch(const Row &row, int64_t base, int64_t n, bool *kp) {
#pragma unroll
    for (int u = 0; u < BC_INFLIGHT; ++u) {  // rows past n test row n - 1 (in bounds, no branch) and drop it
        const int64_t r = base + (int64_t)u * 32;
        kp[u] = row.keep(r < n ? r : n - 1) && r < n;
    }
}
// The keyed pass: the first tested column of all BC_INFLIGHT rows is loaded
// before any row is tested, since a test's early exit would otherwise keep
// the next row's load from being issued ahead of it.
__device__ __forceinline__ void keep_batch(const SemiJoinRow &row, int64_t base, int64_t n, bool *kp) {
    const int32_t *first = row.first_column();
    int32_t v[BC_INFLIGHT];
#pragma unroll
    for (int u = 0; u < BC_INFLIGHT; ++u) {
        const int64_t r = base + (int64_t)u * 32;
        v[u] = first[r < n ? r : n - 1];
    }
#pragma unroll
    for (int u = 0; u < BC_INFLIGHT; ++u) {
        const int64_t r = base + (int64_t)u * 32;
        kp[u] = r < n && row.keep_given(r, v[u]);
    }
}
constexpr int BC_STEP = 1024;      // rows per warp step (32 keep words)
constexpr int BC_DRAW = 8;         // steps per draw from the counter
constexpr int BC_CHUNK = BC_THREADS;  // steps scanned per round of phase C
constexpr int BC_TICKET = 32;      // step counter's word in the control block
constexpr size_t BC_CTL_BYTES = 256;
constexpr int64_t BC_MIN_ROWS = (int64_t)1 << 18;  // below this, the single-pass kernel

struct BcScratch {
    uint32_t *bits;      // 32 keep words per step
    uint32_t *cnt;       // kept rows per step
    unsigned *ctl;       // [1] grid barrier, [BC_TICKET] step counter
    unsigned *cta_tot;   // kept rows per CTA range
    int *err;
    int64_t steps;
};

template <class Row>
__global__ void __launch_bounds__(BC_THREADS, 3)
k_compact_bitmap(Row row, int64_t n, int k_out, OutCols out, int64_t cap, int64_t *__restrict__ d_rows,
                 int64_t *__restrict__ h_rows, BcScratch sc, uint32_t *__restrict__ mm) {
    __shared__ uint16_t s_stage[BC_WARPS][BC_STEP];
    __shared__ uint32_t s_cnt[BC_CHUNK], s_off[BC_CHUNK];
    __shared__ unsigned s_red[BC_WARPS];
    __shared__ unsigned long long s_pre[BC_WARPS], s_all[BC_WARPS];
    __shared__ long long s_base;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per = (sc.steps + gridDim.x - 1) / gridDim.x;  // CTA c owns steps [c per, (c+1) per)

    // ---- phase A: keep words and counts per step
    {
        unsigned *ticket = sc.ctl + BC_TICKET;
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(ticket, (unsigned)BC_DRAW);
        t = __shfl_sync(0xffffffffu, t, 0);
        unsigned k = 0;
        while ((int64_t)(t + k) < sc.steps) {
            const int64_t step = (int64_t)t + k;
            unsigned nxt = 0;
            if (lane == 0 && k + 1 == (unsigned)BC_DRAW) nxt = atomicAdd(ticket, (unsigned)BC_DRAW);
            const int64_t base = step * BC_STEP + lane;
            uint32_t word = 0;
            unsigned c = 0;
#pragma unroll 1
            for (int w0 = 0; w0 < 32; w0 += BC_INFLIGHT) {
                bool kp[BC_INFLIGHT];
                keep_batch(row, base + (int64_t)w0 * 32, n, kp);
#pragma unroll
                for (int u = 0; u < BC_INFLIGHT; ++u) {
                    const unsigned b = __ballot_sync(0xffffffffu, kp[u]);
                    if ((int)lane == w0 + u) word = b;
                    c += __popc(b);
                }
            }
            __stcg(sc.bits + step * 32 + lane, word);
            if (lane == 0) {
                __stcg(sc.cnt + step, c);
                if (c) atomicAdd(sc.cta_tot + step / per, c);
            }
            if (++k == (unsigned)BC_DRAW) {
                t = __shfl_sync(0xffffffffu, nxt, 0);
                k = 0;
            }
        }
    }
    if (!grid_barrier(sc.ctl + 1, gridDim.x, sc.err)) return;

    // ---- phase C: this range's offset, then ordered expansion
    const int64_t r0 = min((int64_t)blockIdx.x * per, sc.steps), r1 = min(r0 + per, sc.steps);
    const unsigned mine = __ldcg(sc.cta_tot + blockIdx.x);
    unsigned long long pre = 0, all = 0;
    for (unsigned c = threadIdx.x; c < gridDim.x; c += BC_THREADS) {
        const unsigned v = __ldcg(sc.cta_tot + c);
        all += v;
        if (c < blockIdx.x) pre += v;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        pre += __shfl_xor_sync(0xffffffffu, pre, d);
        all += __shfl_xor_sync(0xffffffffu, all, d);
    }
    if (lane == 0) {
        s_pre[warp] = pre;
        s_all[warp] = all;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long p = 0, a = 0;
        for (int w = 0; w < BC_WARPS; ++w) {
            p += s_pre[w];
            a += s_all[w];
        }
        s_base = (long long)p;
        if (blockIdx.x == 0) {
            *d_rows = (int64_t)a;
            *h_rows = (int64_t)a;
        }
    }
    __syncthreads();
    if (mine == 0) return;
    uint32_t lo[TID_MAX_COLS], hi[TID_MAX_COLS];
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        lo[c] = 0xFFFFFFFFu;
        hi[c] = 0u;
    }
    long long run = s_base;
    for (int64_t q0 = r0; q0 < r1; q0 += BC_CHUNK) {
        const int64_t j = q0 + threadIdx.x;
        const unsigned c = j < r1 ? __ldcg(sc.cnt + j) : 0u;
        unsigned x = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += y;
        }
        if (lane == 31) s_red[warp] = x;
        __syncthreads();
        unsigned wb = 0, rt = 0;
        for (int w = 0; w < BC_WARPS; ++w) {
            if (w < (int)warp) wb += s_red[w];
            rt += s_red[w];
        }
        s_cnt[threadIdx.x] = c;
        s_off[threadIdx.x] = wb + x - c;
        __syncthreads();
        uint16_t *stage = s_stage[warp];
        for (int i = 0; i < 32; ++i) {  // warp w expands steps q0 + 32 w .. + 31
            const int li = (int)warp * 32 + i;
            const int64_t step = q0 + li;
            if (step >= r1) break;
            const unsigned sn = s_cnt[li];
            if (sn == 0) continue;
            // keep word w of a step holds rows 32 w + (0..31): lane w stages its word's rows
            uint32_t word = __ldcg(sc.bits + step * 32 + lane);
            const unsigned pc = __popc(word);
            unsigned xo = pc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, xo, d);
                if ((int)lane >= d) xo += y;
            }
            unsigned at = xo - pc;
            while (word) {
                const int b = __ffs(word) - 1;
                stage[at++] = (uint16_t)(lane * 32 + b);
                word &= word - 1;
            }
            __syncwarp();
            const long long o0 = run + s_off[li];
#pragma unroll 4
            for (unsigned e = lane; e < sn; e += 32) {
                int32_t v[TID_MAX_COLS];
                row.values(step * BC_STEP + stage[e], v);
                const long long pos = o0 + e;
#pragma unroll
                for (int cc = 0; cc < TID_MAX_COLS; ++cc) {
                    if (cc < k_out) {
                        if ((unsigned long long)pos < (unsigned long long)cap) out.col[cc][pos] = v[cc];
                        const uint32_t u = (uint32_t)v[cc] ^ 0x80000000u;
                        lo[cc] = min(lo[cc], u);
                        hi[cc] = max(hi[cc], u);
                    }
                }
            }
            __syncwarp();
        }
        run += rt;
        __syncthreads();  // s_red, s_cnt, s_off are reused
    }
    if (mm) merge_bounds(mm, k_out, lo, hi);
}

template <class Row>
int bitmap_grid(unsigned *grid) {
    static unsigned cached = 0;
    if (!cached) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_compact_bitmap<Row>, BC_THREADS, 0) != cudaSuccess ||
            v <= 0)
            return fail(TID_ERR_CUDA, "k_compact_bitmap: no resident CTA");
        cached = (unsigned)(v * sm_count());
    }
    *grid = cached;
    return TID_OK;
}

// Which kernel compacts a long input.  Single pass: a tile's offset comes from
// the decoupled look-back, and profiles show tiles waiting there for their
// predecessors far longer than their own work takes; it serves short inputs
// and bind with tests (its tests are random gathers: two kernels would gather
// them twice, and measured no faster).  Two kernels (filters, distinct rows):
// the test columns are read twice and no CTA waits for another.  Bitmap
// (sparse keeps over the store: the keyed pass): one cooperative launch, the
// kept rows' values read once after the grid barrier.
enum CompactMode { CP_SINGLE, CP_TWO, CP_BITMAP };

template <class Row>
int launch_compact(tid_ctx *ctx, const Row &row, int64_t n, int k_out, const OutCols &out, int64_t cap,
                   int64_t *d_rows, int64_t *h_rows_dev, uint32_t *mm = nullptr, CompactMode mode = CP_TWO) {
    if (n == 0) {
        TID_TRY_CUDA(cudaMemsetAsync(d_rows, 0, sizeof(int64_t), ctx->stream), "memset rows");
        TID_TRY_CUDA(cudaMemsetAsync(h_rows_dev, 0, sizeof(int64_t), ctx->stream), "memset rows");
        return TID_OK;
    }
    if (n >= BC_MIN_ROWS && mode == CP_TWO) {
        static bool opted = false;
        if (!opted) {
            TID_TRY_CUDA(cudaFuncSetAttribute(k_tile_write<Row>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(sizeof(int32_t) * TID_MAX_COLS * CP_TILE)),
                         "k_tile_write smem");
            opted = true;
        }
        const unsigned tiles = (unsigned)ceil_div(n, CP_TILE);
        void *blk = nullptr;
        TID_TRY(dev_alloc(ctx, &blk, sizeof(uint32_t) * 2 * (size_t)tiles + 256));
        uint32_t *counts = (uint32_t *)blk, *offs = counts + tiles;
        int rc = TID_OK;
        k_tile_counts<Row><<<tiles, CP_THREADS, 0, ctx->stream>>>(row, n, counts);
        rc = launch_check("k_tile_counts");
        if (rc == TID_OK) rc = scan_exclusive_u32(ctx, counts, offs, tiles, nullptr);
        if (rc == TID_OK) {
            const size_t smem = sizeof(int32_t) * (size_t)std::max(1, k_out) * CP_TILE;
            k_tile_write<Row><<<tiles, CP_THREADS, smem, ctx->stream>>>(row, n, k_out, out, cap, offs, counts, tiles,
                                                                        d_rows, h_rows_dev, mm);
            rc = launch_check("k_tile_write");
        }
        dev_free(ctx, blk);
        return rc;
    }
    if (n < BC_MIN_ROWS || mode == CP_SINGLE) {
        static bool opted = false;  // staging of up to TID_MAX_COLS columns of a tile
        if (!opted) {
            TID_TRY_CUDA(cudaFuncSetAttribute(k_compact<Row>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)(sizeof(int32_t) * TID_MAX_COLS * CP_TILE)),
                         "k_compact smem");
            opted = true;
        }
        const unsigned tiles = (unsigned)ceil_div(n, CP_TILE);
        Lookback lb{};
        TID_TRY(lookback_scratch(ctx, tiles, &lb));
        const size_t smem = sizeof(int32_t) * (size_t)std::max(1, k_out) * CP_TILE;
        k_compact<Row><<<tiles, CP_THREADS, smem, ctx->stream>>>(row, n, k_out, out, cap, d_rows, h_rows_dev, lb, mm);
        return launch_check("k_compact");
    }
    unsigned grid = 0;
    TID_TRY(bitmap_grid<Row>(&grid));
    const int64_t steps = ceil_div(n, (int64_t)BC_STEP);
    grid = (unsigned)std::min<int64_t>(grid, steps);
    const size_t bits_b = (size_t)steps * 32 * 4, cnt_b = ((size_t)steps * 4 + 255) / 256 * 256;
    const size_t tot_b = (size_t)grid * 4;
    void *blk = nullptr;
    TID_TRY(dev_alloc(ctx, &blk, bits_b + cnt_b + BC_CTL_BYTES + tot_b));
    BcScratch sc{};
    sc.bits = (uint32_t *)blk;
    sc.cnt = (uint32_t *)((char *)blk + bits_b);
    sc.ctl = (unsigned *)((char *)blk + bits_b + cnt_b);
    sc.cta_tot = (unsigned *)((char *)blk + bits_b + cnt_b + BC_CTL_BYTES);
    sc.err = ctx->err_dev;
    sc.steps = steps;
    int rc = TID_OK;
    cudaError_t e = cudaMemsetAsync(sc.ctl, 0, BC_CTL_BYTES + tot_b, ctx->stream);
    if (e != cudaSuccess) rc = fail_cuda(e, "k_compact_bitmap control words");
    if (rc == TID_OK) {
        Row r = row;
        OutCols oc = out;
        void *args[] = {(void *)&r, (void *)&n, (void *)&k_out, (void *)&oc, (void *)&cap, (void *)&d_rows,
                        (void *)&h_rows_dev, (void *)&sc, (void *)&mm};
        e = cudaLaunchCooperativeKernel((const void *)k_compact_bitmap<Row>, dim3(grid), dim3(BC_THREADS), args, 0,
                                        ctx->stream);
        if (e != cudaSuccess) rc = fail_cuda(e, "k_compact_bitmap");
    }
    dev_free(ctx, blk);
    return rc;
}

// Bind with nothing to test (no repeated variable, no predicate): every row is
// kept in index order, so row r is written at r -- a plain gather, no
// compaction -- with the column bounds of the output.
__global__ void __launch_bounds__(256) k_bind_gather(BindRow row, int64_t n, OutCols out, uint32_t *__restrict__ mm,
                                                     int64_t *__restrict__ d_rows, int64_t *__restrict__ h_rows) {
    uint32_t lo[TID_MAX_COLS], hi[TID_MAX_COLS];
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        lo[c] = 0xFFFFFFFFu;
        hi[c] = 0u;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_iter = ceil_div(n, stride) * stride;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_iter; r += stride) {
        if (r < n) {
            int32_t v[TID_MAX_COLS];
            row.values(r, v);
#pragma unroll
            for (int c = 0; c < TID_MAX_COLS; ++c) {
                if (c < row.k) {
                    out.col[c][r] = v[c];
                    const uint32_t u = (uint32_t)v[c] ^ 0x80000000u;
                    lo[c] = min(lo[c], u);
                    hi[c] = max(hi[c], u);
                }
            }
        }
    }
    if (mm) merge_bounds(mm, row.k, lo, hi);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_rows = n;
        *h_rows = n;
    }
}

// ---- exclusive scan of uint32 (look-back) --------------------------------------

constexpr int SC_THREADS = 256, SC_ITEMS = 16, SC_TILE = SC_THREADS * SC_ITEMS;
static_assert(SC_ITEMS == 16, "k_scan_u32 splits tile positions as (e >> 4, e & 15)");

// Exclusive scan of one 4096-item tile; the tile's first output is `prefix`
// (from offs[tile] when offs is given, else by decoupled look-back -- used for a
// single tile, where nothing waits).  total_out: the sum of all items.
__global__ void __launch_bounds__(SC_THREADS)
k_scan_u32(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
           unsigned long long *__restrict__ total_out, Lookback lb, const uint32_t *__restrict__ offs) {
    __shared__ unsigned s_tile;
    __shared__ uint32_t s_w[SC_THREADS / 32];
    __shared__ long long s_prefix;
    // the tile, thread-blocked (thread t's items at t * 17 .. t * 17 + 15: the
    // odd stride keeps a warp's blocked reads on distinct banks); global loads
    // and stores go through it striped, so they are coalesced
    __shared__ uint32_t s_t[SC_THREADS * (SC_ITEMS + 1)];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = offs ? blockIdx.x : lb_ticket(lb);
    __syncthreads();
    const unsigned tile = s_tile;
    if (!offs && tile >= lb.num_tiles) return;
    const int64_t base0 = (int64_t)tile * SC_TILE;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        const int e = i * SC_THREADS + threadIdx.x;
        s_t[(e >> 4) * (SC_ITEMS + 1) + (e & 15)] = base0 + e < n ? in[base0 + e] : 0u;
    }
    __syncthreads();
    uint32_t v[SC_ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        v[i] = s_t[threadIdx.x * (SC_ITEMS + 1) + i];
        sum += v[i];
    }
    uint32_t x = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((int)lane >= d) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < SC_THREADS / 32 ? s_w[lane] : 0u;
        uint32_t y = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t z = __shfl_up_sync(0xffffffffu, y, d);
            if ((int)lane >= d) y += z;
        }
        if (lane < SC_THREADS / 32) s_w[lane] = y - w;
        const uint32_t total = __shfl_sync(0xffffffffu, y, 31);
        if (offs) {
            if (lane == 0) s_prefix = offs[tile];
        } else {
            const long long excl = lb_exclusive_prefix(lb, tile, total);
            if (lane == 0) {
                s_prefix = excl;
                if (tile == lb.num_tiles - 1 && excl >= 0 && total_out) *total_out = excl + total;
            }
        }
    }
    __syncthreads();
    if (s_prefix < 0) return;
    uint32_t run = (uint32_t)s_prefix + s_w[warp] + (x - sum);
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        s_t[threadIdx.x * (SC_ITEMS + 1) + i] = run;
        run += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        const int e = i * SC_THREADS + threadIdx.x;
        if (base0 + e < n) out[base0 + e] = s_t[(e >> 4) * (SC_ITEMS + 1) + (e & 15)];
    }
}

// sums[t] = sum of the items of tile t (SC_TILE items)
__global__ void __launch_bounds__(SC_THREADS) k_tile_sums(const uint32_t *__restrict__ in, int64_t n,
                                                          uint32_t *__restrict__ sums) {
    __shared__ uint32_t s_w[SC_THREADS / 32];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SC_TILE;
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {  // striped: coalesced
        const int64_t j = base + i * SC_THREADS + threadIdx.x;
        sum += j < n ? in[j] : 0u;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0) s_w[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SC_THREADS / 32; ++w) t += s_w[w];
        sums[blockIdx.x] = t;
    }
}

}  // namespace

int scan_exclusive_u32(tid_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n,
                       unsigned long long *total_dev) {
    if (n == 0) {
        if (total_dev) TID_TRY_CUDA(cudaMemsetAsync(total_dev, 0, 8, ctx->stream), "memset");
        return TID_OK;
    }
    const unsigned tiles = (unsigned)ceil_div(n, SC_TILE);
    if (tiles == 1) {  // one tile: nothing to wait for
        Lookback lb{};
        TID_TRY(lookback_scratch(ctx, 1, &lb));
        k_scan_u32<<<1, SC_THREADS, 0, ctx->stream>>>(in, out, n, total_dev, lb, nullptr);
        return launch_check("k_scan_u32");
    }
    // reduce, scan the tile sums (recursively), scan each tile from its offset:
    // no tile waits for another
    uint32_t *sums = nullptr;
    TID_TRY(dev_alloc(ctx, (void **)&sums, sizeof(uint32_t) * 2 * (size_t)tiles + 256));
    uint32_t *offs = sums + tiles;
    k_tile_sums<<<tiles, SC_THREADS, 0, ctx->stream>>>(in, n, sums);
    int rc = launch_check("k_tile_sums");
    if (rc == TID_OK) rc = scan_exclusive_u32(ctx, sums, offs, tiles, total_dev);
    if (rc == TID_OK) {
        k_scan_u32<<<tiles, SC_THREADS, 0, ctx->stream>>>(in, out, n, nullptr, Lookback{}, offs);
        rc = launch_check("k_scan_u32");
    }
    dev_free(ctx, sums);
    return rc;
}

int compact_bind(tid_ctx *ctx, const tid_store *st, const tid_pattern &pat, const int32_t *idx, int64_t n,
                 const Pred *preds, int n_preds, tid_set *out, uint32_t *mm) {
    BindRow r{};
    r.S = st->s;
    r.P = st->p;
    r.O = st->o;
    r.idx = idx;
    r.k = out->k;
    const int8_t var[3] = {pat.var[0], pat.var[1], pat.var[2]};
    r.need = (var[0] >= 0 ? 1 : 0) | (var[1] >= 0 ? 2 : 0) | (var[2] >= 0 ? 4 : 0);
    for (int c = 0; c < out->k; ++c) {
        r.src[c] = -1;
        for (int j = 0; j < 3; ++j)
            if (var[j] == out->vars[c]) {
                r.src[c] = (int8_t)j;
                break;
            }
    }
    r.n_eq = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (var[a] >= 0 && var[a] == var[b]) {
                r.eq_a[r.n_eq] = (int8_t)a;
                r.eq_b[r.n_eq] = (int8_t)b;
                r.n_eq++;
            }
    r.n_preds = n_preds;
    for (int q = 0; q < n_preds; ++q) r.preds[q] = preds[q];
    OutCols oc{};
    for (int c = 0; c < out->k; ++c) oc.col[c] = out->col[c];
    if (n > 0 && r.n_eq == 0 && r.n_preds == 0 && n <= out->cap) {
        k_bind_gather<<<grid_for(n, 256, 8), 256, 0, ctx->stream>>>(r, n, oc, mm, out->d_rows, out->slot.dev);
        return launch_check("k_bind_gather");
    }
    return launch_compact(ctx, r, n, out->k, oc, out->cap, out->d_rows, out->slot.dev, mm, CP_SINGLE);
}

int compact_semijoin(tid_ctx *ctx, const tid_store *st, int fixed_slot, int32_t fixed_val, int key_slot,
                     const int32_t *table, int tbits, const int8_t *src, tid_set *out) {
    SemiJoinRow r{};
    r.S = st->s;
    r.P = st->p;
    r.O = st->o;
    r.fixed_slot = fixed_slot;
    r.fixed_val = fixed_val;
    r.key_slot = key_slot;
    r.table = table;
    r.tbits = tbits;
    r.k = out->k;
    r.need = (fixed_slot >= 0 ? 1 << fixed_slot : 0) | (1 << key_slot);
    for (int c = 0; c < out->k; ++c) {
        r.src[c] = src[c];
        r.need |= 1 << src[c];
    }
    OutCols oc{};
    for (int c = 0; c < out->k; ++c) oc.col[c] = out->col[c];
    return launch_compact(ctx, r, st->n, out->k, oc, out->cap, out->d_rows, out->slot.dev, nullptr, CP_BITMAP);
}

int compact_filter(tid_ctx *ctx, const tid_set *in, int64_t n, const Pred *preds, int n_preds, tid_set *out) {
    FilterRow r{};
    r.k = in->k;
    for (int c = 0; c < in->k; ++c) r.col[c] = in->col[c];
    r.n_preds = n_preds;
    for (int q = 0; q < n_preds; ++q) r.preds[q] = preds[q];
    OutCols oc{};
    for (int c = 0; c < out->k; ++c) oc.col[c] = out->col[c];
    return launch_compact(ctx, r, n, out->k, oc, out->cap, out->d_rows, out->slot.dev);
}

int compact_unique(tid_ctx *ctx, const int32_t *const *cols, int k, const int32_t *perm, int64_t n,
                   tid_set *out) {
    UniqueRow r{};
    r.k = k;
    for (int c = 0; c < k; ++c) r.col[c] = cols[c];
    r.perm = perm;
    OutCols oc{};
    for (int c = 0; c < out->k; ++c) oc.col[c] = out->col[c];
    return launch_compact(ctx, r, n, out->k, oc, out->cap, out->d_rows, out->slot.dev);
}

int compact_unique_packed(tid_ctx *ctx, const void *keys, bool wide, int k, int64_t n, const PackSpec &ps,
                          tid_set *out) {
    OutCols oc{};
    for (int c = 0; c < out->k; ++c) oc.col[c] = out->col[c];
    if (wide) {
        PackedUniqueRow<unsigned long long> r{(const unsigned long long *)keys, ps, k};
        return launch_compact(ctx, r, n, out->k, oc, out->cap, out->d_rows, out->slot.dev);
    }
    PackedUniqueRow<uint32_t> r{(const uint32_t *)keys, ps, k};
    return launch_compact(ctx, r, n, out->k, oc, out->cap, out->d_rows, out->slot.dev);
}

}  // namespace tid
