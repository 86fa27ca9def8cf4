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

// Row sources write v[0..k) and say whether the row is kept.  Column loops run
// to TID_MAX_COLS with a guard so v[] stays in registers.

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
    __device__ __forceinline__ bool load(int64_t r, int32_t *v) const {
        const int64_t t = idx[r];
        // only the variable slots are read: a bound slot holds the key itself
        const int32_t t0 = (need & 1) ? S[t] : 0;
        const int32_t t1 = (need & 2) ? P[t] : 0;
        const int32_t t2 = (need & 4) ? O[t] : 0;
        bool ok = true;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            if (e < n_eq) {
                const int32_t a = eq_a[e] == 0 ? t0 : (eq_a[e] == 1 ? t1 : t2);
                const int32_t b = eq_b[e] == 0 ? t0 : (eq_b[e] == 1 ? t1 : t2);
                ok = ok && a == b;
            }
        }
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) v[c] = src[c] == 0 ? t0 : (src[c] == 1 ? t1 : t2);
        return ok && preds_ok(preds, n_preds, v);
    }
};

struct FilterRow {
    const int32_t *col[TID_MAX_COLS];
    int k;
    Pred preds[MAX_PREDS];
    int n_preds;
    __device__ __forceinline__ bool load(int64_t r, int32_t *v) const {
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) v[c] = col[c][r];
        return preds_ok(preds, n_preds, v);
    }
};

struct UniqueRow {  // rows in perm order; keep the first of each run of equal rows
    const int32_t *col[TID_MAX_COLS];
    const int32_t *perm;  // may be null (rows already in order)
    int k;
    __device__ __forceinline__ bool load(int64_t r, int32_t *v) const {
        const int64_t a = perm ? perm[r] : r;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) v[c] = col[c][a];
        if (r == 0) return true;
        const int64_t b = perm ? perm[r - 1] : r - 1;
        bool same = true;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) same = same && col[c][b] == v[c];
        return !same;
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
    uint32_t tmask;             // table size - 1 (a power of two)
    int k;
    int8_t src[TID_MAX_COLS];   // slot giving output column c
    __device__ __forceinline__ const int32_t *column(int slot) const { return slot == 0 ? S : (slot == 1 ? P : O); }
    // the fixed and the key column first; the other columns only for rows that pass
    __device__ __forceinline__ bool load(int64_t r, int32_t *v) const {
        if (fixed_slot >= 0 && column(fixed_slot)[r] != fixed_val) return false;
        const int32_t key = column(key_slot)[r];
        if (key == 0) return false;
        uint32_t h = ((uint32_t)key * 0x9E3779B1u) & tmask;
        bool found = false;
        for (uint32_t probe = 0; probe <= tmask; ++probe) {  // the table is at most half full
            const int32_t e = __ldg(table + h);
            if (e == key) {
                found = true;
                break;
            }
            if (e == 0) break;
            h = (h + 1) & tmask;
        }
        if (!found) return false;
        const int32_t t0 = (need & 1) ? S[r] : 0;
        const int32_t t1 = (need & 2) ? P[r] : 0;
        const int32_t t2 = (need & 4) ? O[r] : 0;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < k) v[c] = src[c] == 0 ? t0 : (src[c] == 1 ? t1 : t2);
        return true;
    }
};

template <typename K>
struct PackedUniqueRow {  // sorted packed keys; keep the first of each run of equal keys
    const K *keys;
    PackSpec ps;
    int k;
    __device__ __forceinline__ bool load(int64_t r, int32_t *v) const {
        const K key = keys[r];
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c < k) {
                const uint32_t f = ps.mask[c] ? (uint32_t)((key >> ps.shift[c]) & ps.mask[c]) : 0u;
                v[c] = (int32_t)((f + ps.min[c]) ^ 0x80000000u);
            }
        }
        return r == 0 || keys[r - 1] != key;
    }
};

template <class Row>
__global__ void __launch_bounds__(CP_THREADS)
k_compact(Row row, int64_t n, int k_out, OutCols out, int64_t cap, int64_t *__restrict__ d_rows,
          int64_t *__restrict__ h_rows, Lookback lb, uint32_t *__restrict__ mm) {
    __shared__ unsigned s_tile;
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
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) {
        const int64_t r = base + j * CP_THREADS + threadIdx.x;
        int32_t v[TID_MAX_COLS];
        const bool kp = r < n && row.load(r, v);
        keep |= (unsigned)kp << j;
        const unsigned b = __ballot_sync(0xffffffffu, kp);
        wpre[j] = __popc(b & lt);
        if (lane == 0) s_off[j * CP_WARPS + warp] = __popc(b);
    }
    __syncthreads();
    if (warp == 0) {
        // 64 (item, warp) counts in order; each lane scans two consecutive entries
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
        const unsigned total = __shfl_sync(0xffffffffu, x, 31);
        const long long excl = lb_exclusive_prefix(lb, tile, total);
        if (lane == 0) {
            s_prefix = excl;
            if (tile == lb.num_tiles - 1 && excl >= 0) {
                *d_rows = excl + total;
                *h_rows = excl + total;
            }
        }
    }
    __syncthreads();
    const long long prefix = s_prefix;
    if (prefix < 0) return;
    uint32_t lo[TID_MAX_COLS], hi[TID_MAX_COLS];
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        lo[c] = 0xFFFFFFFFu;
        hi[c] = 0u;
    }
#pragma unroll
    for (int j = 0; j < CP_ITEMS; ++j) {
        if (!((keep >> j) & 1u)) continue;
        const int64_t r = base + j * CP_THREADS + threadIdx.x;
        int32_t v[TID_MAX_COLS];
        row.load(r, v);  // second read of a kept row (cached in L1/L2)
        const long long pos = prefix + s_off[j * CP_WARPS + warp] + wpre[j];
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c < k_out) {
                if (pos < cap) out.col[c][pos] = v[c];
                const uint32_t u = (uint32_t)v[c] ^ 0x80000000u;
                lo[c] = min(lo[c], u);
                hi[c] = max(hi[c], u);
            }
        }
    }
    if (mm) {  // column bounds of the kept rows
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c < k_out) {
                uint32_t a = lo[c], b = hi[c];
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    a = min(a, __shfl_xor_sync(0xffffffffu, a, d));
                    b = max(b, __shfl_xor_sync(0xffffffffu, b, d));
                }
                if (lane == 0 && a <= b) {
                    atomicMin(mm + c, a);
                    atomicMax(mm + TID_MAX_COLS + c, b);
                }
            }
        }
    }
}

template <class Row>
int launch_compact(tid_ctx *ctx, const Row &row, int64_t n, int k_out, const OutCols &out, int64_t cap,
                   int64_t *d_rows, int64_t *h_rows_dev, uint32_t *mm = nullptr) {
    if (n == 0) {
        TID_TRY_CUDA(cudaMemsetAsync(d_rows, 0, sizeof(int64_t), ctx->stream), "memset rows");
        TID_TRY_CUDA(cudaMemsetAsync(h_rows_dev, 0, sizeof(int64_t), ctx->stream), "memset rows");
        return TID_OK;
    }
    const unsigned tiles = (unsigned)ceil_div(n, CP_TILE);
    Lookback lb{};
    TID_TRY(lookback_scratch(ctx, tiles, &lb));
    k_compact<Row><<<tiles, CP_THREADS, 0, ctx->stream>>>(row, n, k_out, out, cap, d_rows, h_rows_dev, lb, mm);
    return launch_check("k_compact");
}

// ---- exclusive scan of uint32 (look-back) --------------------------------------

constexpr int SC_THREADS = 256, SC_ITEMS = 16, SC_TILE = SC_THREADS * SC_ITEMS;

__global__ void __launch_bounds__(SC_THREADS)
k_scan_u32(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int64_t n,
           unsigned long long *__restrict__ total_out, Lookback lb) {
    __shared__ unsigned s_tile;
    __shared__ uint32_t s_w[SC_THREADS / 32];
    __shared__ long long s_prefix;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = lb_ticket(lb);
    __syncthreads();
    const unsigned tile = s_tile;
    if (tile >= lb.num_tiles) return;
    // blocked: thread t owns items base + t*16 .. +15
    const int64_t base = (int64_t)tile * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
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
        const long long excl = lb_exclusive_prefix(lb, tile, total);
        if (lane == 0) {
            s_prefix = excl;
            if (tile == lb.num_tiles - 1 && excl >= 0 && total_out) *total_out = excl + total;
        }
    }
    __syncthreads();
    if (s_prefix < 0) return;
    uint32_t run = (uint32_t)s_prefix + s_w[warp] + (x - sum);
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
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
    Lookback lb{};
    TID_TRY(lookback_scratch(ctx, tiles, &lb));
    k_scan_u32<<<tiles, SC_THREADS, 0, ctx->stream>>>(in, out, n, total_dev, lb);
    return launch_check("k_scan_u32");
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
    return launch_compact(ctx, r, n, out->k, oc, out->cap, out->d_rows, out->slot.dev, mm);
}

int compact_semijoin(tid_ctx *ctx, const tid_store *st, int fixed_slot, int32_t fixed_val, int key_slot,
                     const int32_t *table, uint32_t tmask, const int8_t *src, tid_set *out) {
    SemiJoinRow r{};
    r.S = st->s;
    r.P = st->p;
    r.O = st->o;
    r.fixed_slot = fixed_slot;
    r.fixed_val = fixed_val;
    r.key_slot = key_slot;
    r.table = table;
    r.tmask = tmask;
    r.k = out->k;
    r.need = (fixed_slot >= 0 ? 1 << fixed_slot : 0) | (1 << key_slot);
    for (int c = 0; c < out->k; ++c) {
        r.src[c] = src[c];
        r.need |= 1 << src[c];
    }
    OutCols oc{};
    for (int c = 0; c < out->k; ++c) oc.col[c] = out->col[c];
    return launch_compact(ctx, r, st->n, out->k, oc, out->cap, out->d_rows, out->slot.dev);
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
