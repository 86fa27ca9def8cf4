// K5 / K6: inner join of two tuple sets on all shared variables.
//
// Section 4.2 joins subquery result vectors by copying the related terms into
// key vectors, sorting them, and running a merge-join that returns pairs of
// matching positions, from which the remaining values are gathered; the
// relationship table lists the nine S/P/O position pairings a shared term can
// take, which here are simply the columns of the shared variables.
//
// Both algorithms follow the same three phases (the two-phase output sizing
// of He et al. that the paper cites): count matches per row, exclusive-scan
// the counts (one synchronisation reads the total to size the output), then
// write every output row with one thread -- an output row finds its left row
// by binary search over the scanned counts, so a key with millions of matches
// is spread over as many threads (no per-row serial loops).
//
//  * sort-merge: both sides ordered by the key (free when the key columns are
//    a prefix of a canonical set's column order; else a radix-sorted
//    permutation); per left row, lower/upper bound in the right keys.
//  * hash: the smaller side is grouped by key in an open-addressing table
//    (key -> [start, count) into a grouped row array, built with CAS inserts,
//    a scan and a scatter); the other side probes it.  A table of at most
//    2048 slots is copied into shared memory by every probing CTA.
// A key value 0 (unbound) never matches.  The output is sorted to canonical
// order unless it is written in that order already (both inputs lead with the
// shared variables); a join of two sets is a set, so no duplicate removal is
// needed.
//
// Left outer join (OPTIONAL; the library the paper used also offered outer and
// left joins, Section 4.2): sort-merge only; a left row without a match counts
// as one output row (its right range marked empty) and is written with the
// right side's other columns 0 (unbound).

#include <algorithm>

#include "lookback.cuh"
#include "ops.cuh"

namespace tid {

int set_rows_const(tid_set *set, int64_t n);

namespace {

struct Cols {
    const int32_t *c[TID_MAX_COLS];
};
struct MCols {
    int32_t *c[TID_MAX_COLS];
};

// Column loops run to TID_MAX_COLS with a guard: constant indices keep the
// column pointers in registers (a loop bounded by nk would copy the parameter
// arrays to local memory).
__device__ __forceinline__ int cmp_rows(const Cols &A, int64_t a, const Cols &B, int64_t b, int nk) {
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        if (c >= nk) break;
        const int32_t x = A.c[c][a], y = B.c[c][b];
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

__device__ __forceinline__ bool has_zero(const Cols &A, int64_t a, int nk) {
    bool z = false;
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c)
        if (c < nk) z = z || A.c[c][a] == 0;
    return z;
}

// Output row o of a join: L's kl columns of row lr, then R's other columns of
// row rr (rr < 0: unbound, 0).  outL / outR point at the output columns of
// each part, so every index here is a constant.
__device__ __forceinline__ void write_out(const Cols &L, int kl, const Cols &Rrest, int nrest, int64_t lr, int64_t rr,
                                          const MCols &outL, const MCols &outR, int64_t o) {
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c)
        if (c < kl) outL.c[c][o] = L.c[c][lr];
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c)
        if (c < nrest) outR.c[c][o] = rr < 0 ? 0 : Rrest.c[c][rr];
}

__device__ __forceinline__ void block_add_u64(unsigned long long v, unsigned long long *total) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// ---- sort-merge --------------------------------------------------------------
// [lo, hi) of the right keys equal to left key row l, searched inside [a0, b0)
__device__ __forceinline__ void eq_range(const Cols &RK, const Cols &LK, int64_t l, int nk, int64_t a0, int64_t b0,
                                         int64_t *lo, int64_t *hi) {
    int64_t a = a0, b = b0;  // lower bound
    while (a < b) {
        const int64_t m = (a + b) >> 1;
        if (cmp_rows(RK, m, LK, l, nk) < 0) a = m + 1;
        else b = m;
    }
    int64_t a2 = a, b2 = b0;  // upper bound
    while (a2 < b2) {
        const int64_t m = (a2 + b2) >> 1;
        if (cmp_rows(RK, m, LK, l, nk) <= 0) a2 = m + 1;
        else b2 = m;
    }
    *lo = a;
    *hi = a2;
}

// The left keys are sorted, so the right range of every left row of a warp
// lies between the lower bound of the warp's first row and the upper bound of
// its last: two searches over all of R per warp (lanes 0 and 31), then each
// lane searches only that bracket (a few cache lines, not DRAM at every level).
// first / last: the warp's first and last left rows (valid, first <= last).
__device__ __forceinline__ void warp_bracket(const Cols &RK, const Cols &LK, int nk, int64_t nr, int64_t first,
                                             int64_t last, int64_t *a0, int64_t *b0) {
    const unsigned lane = threadIdx.x & 31;
    int64_t lo = 0, hi = nr;
    if (lane == 0) {
        int64_t x, y;
        eq_range(RK, LK, first, nk, 0, nr, &x, &y);
        lo = x;
    } else if (lane == 31) {
        int64_t x, y;
        eq_range(RK, LK, last, nk, 0, nr, &x, &y);
        hi = y;
    }
    *a0 = __shfl_sync(0xffffffffu, lo, 0);
    *b0 = __shfl_sync(0xffffffffu, hi, 31);
}



// per left row: [lo, hi) of equal keys in the sorted right keys
constexpr uint32_t NO_MATCH = 0xFFFFFFFFu;  // left outer join: a left row written once, padded

__global__ void k_sm_count(Cols LK, int64_t nl, Cols RK, int64_t nr, int nk, bool left, uint32_t *__restrict__ cnt,
                           uint32_t *__restrict__ lo_out, unsigned long long *__restrict__ total) {
    unsigned long long acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_iter = ceil_div(nl, stride) * stride;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n_iter; l += stride) {
        const int64_t w0 = l - (threadIdx.x & 31);  // the warp's rows: w0 .. w0 + 31
        int64_t a0 = 0, b0 = nr;
        if (w0 < nl) warp_bracket(RK, LK, nk, nr, w0, min(w0 + 31, nl - 1), &a0, &b0);
        if (l < nl) {
            uint32_t c = 0, lo = 0;
            if (!has_zero(LK, l, nk)) {
                int64_t a, a2;
                eq_range(RK, LK, l, nk, a0, b0, &a, &a2);
                lo = (uint32_t)a;
                c = (uint32_t)(a2 - a);
            }
            if (left && c == 0) {
                c = 1;
                lo = NO_MATCH;
            }
            cnt[l] = c;
            lo_out[l] = lo;
            acc += c;
        }
    }
    block_add_u64(acc, total);  // once per warp: one address takes these atomics one at a time
}

// Output rows of probe rows: probe row l's matches are written at off[l] ..
// off[l + 1] - 1 (off the exclusive scan of the counts, total their sum).
// Load-balanced search (the merge-path partition of Odeh et al. applied to
// the sequences of row starts and output rows): CTA t takes items [t T, (t+1) T)
// of their merged order (row l before output o when off[l] <= o), i.e. some
// probe rows and the output rows next to them -- at most T items in all, so
// neither a long run of rows without matches nor one row with millions of
// matches makes a CTA's work unbounded.  The CTA stages its rows' offsets in
// shared memory and each output row finds its probe row there by binary
// search; consecutive output rows go to consecutive threads (coalesced
// stores).
constexpr int JW_THREADS = 256;
constexpr int JW_ITEMS = 8;
constexpr int JW_TILE = JW_THREADS * JW_ITEMS;

// rows among the first d items of the merged order
__device__ __forceinline__ int64_t jw_split(const uint32_t *__restrict__ off, int64_t nl, int64_t total, int64_t d) {
    int64_t lo = max((int64_t)0, d - total), hi = min(d, nl);
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)off[mid] <= d - 1 - mid) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void join_row(const uint32_t *__restrict__ lo, const int32_t *__restrict__ lperm,
                                         const int32_t *__restrict__ rmap, const int32_t *__restrict__ rperm,
                                         const Cols &L, int kl, const Cols &Rrest, int nrest, const MCols &outL,
                                         const MCols &outR, bool left_is_probe, int64_t l, uint32_t lol, int64_t k,
                                         int64_t o) {
    if (lol == NO_MATCH) {  // left outer join: the left row alone, right columns unbound
        write_out(L, kl, Rrest, nrest, lperm ? lperm[l] : l, -1, outL, outR, o);
        return;
    }
    const int64_t j = (int64_t)lol + k;
    int64_t lr, rr;
    if (left_is_probe) {
        lr = lperm ? lperm[l] : l;
        rr = rmap ? rmap[j] : j;
        if (rperm) rr = rperm[rr];
    } else {  // hash join built on the left: "l" walks right rows, j indexes grouped left rows
        rr = l;
        lr = rmap[j];
    }
    write_out(L, kl, Rrest, nrest, lr, rr, outL, outR, o);
}

__global__ void __launch_bounds__(JW_THREADS) k_join_write(const uint32_t *__restrict__ off, int64_t nl,
                                                           const uint32_t *__restrict__ lo,
                                                           const int32_t *__restrict__ lperm,
                                                           const int32_t *__restrict__ rmap,
                                                           const int32_t *__restrict__ rperm, int64_t total, Cols L,
                                                           int kl, Cols Rrest, int nrest, MCols outL, MCols outR,
                                                           bool left_is_probe) {
    __shared__ uint32_t s_off[JW_TILE + 1];  // off[rb .. r1 - 1]
    __shared__ int64_t s_r[2];
    const int64_t d0 = (int64_t)blockIdx.x * JW_TILE, d1 = min(d0 + JW_TILE, nl + total);
    if (threadIdx.x < 2) s_r[threadIdx.x] = jw_split(off, nl, total, threadIdx.x == 0 ? d0 : d1);
    __syncthreads();
    const int64_t r0 = s_r[0], r1 = s_r[1];
    const int64_t o0 = d0 - r0, o1 = d1 - r1;
    if (o0 >= o1) return;  // only rows here
    // the output rows [o0, o1) belong to rows rb .. r1 - 1: row r0 - 1 precedes
    // output o0 in the merged order (off[r0 - 1] <= o0), row r1 follows o1 - 1
    const int64_t rb = r0 > 0 ? r0 - 1 : 0;
    const int nr = (int)(r1 - rb);
    for (int i = threadIdx.x; i < nr; i += JW_THREADS) s_off[i] = off[rb + i];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < JW_ITEMS; ++q) {
        const int64_t o = o0 + q * JW_THREADS + threadIdx.x;
        if (o >= o1) break;
        // last i with s_off[i] <= o.  First guess: rows of one match each
        // (the common case) put output o at row o - s_off[0] of the tile.
        int a = (int)min((int64_t)(nr - 1), o - (int64_t)s_off[0]);
        if (!((int64_t)s_off[a] <= o && (a + 1 == nr || (int64_t)s_off[a + 1] > o))) {
            a = 0;
            int b = nr;
            while (b - a > 1) {
                const int m = (a + b) >> 1;
                if ((int64_t)s_off[m] <= o) a = m;
                else b = m;
            }
        }
        const int64_t l = rb + a;
        join_row(lo, lperm, rmap, rperm, L, kl, Rrest, nrest, outL, outR, left_is_probe, l, lo[l], o - s_off[a], o);
    }
}

// Single-pass sort-merge join of inputs that both lead with the key (so they
// are sorted by it) when one side holds only key columns: then every row of
// the other side matches at most one row, the output has at most
// (|other side|, + |L| for a left join) rows, and it can be written without a
// separate count pass.  A CTA takes a tile of MJ_TILE left rows (tickets in
// order); each thread finds the matching range of its rows in R (two binary
// searches), the block scans the counts, the decoupled look-back gives the
// tile's first output row, and the CTA writes its output rows in order --
// an output row finds its left row by binary search over the tile's scanned
// counts in shared memory, so a key with many matches is spread over all the
// CTA's threads.  The output is canonical as written.
constexpr int MJ_THREADS = 256;
constexpr int MJ_ITEMS = 4;
constexpr int MJ_TILE = MJ_THREADS * MJ_ITEMS;

__global__ void __launch_bounds__(MJ_THREADS)
k_merge_join(Cols LK, int64_t nl, Cols RK, int64_t nr, int nk, bool left, Cols L, int kl, Cols Rrest, int nrest,
             MCols outL, MCols outR, int64_t cap, int64_t *__restrict__ d_rows, int64_t *__restrict__ h_rows,
             Lookback lb) {
    __shared__ uint32_t s_excl[MJ_TILE + 1], s_lo[MJ_TILE];
    __shared__ uint32_t s_wsum[MJ_THREADS / 32];
    __shared__ unsigned s_tile;
    __shared__ long long s_prefix;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = lb_ticket(lb);
    __syncthreads();
    const unsigned tile = s_tile;
    if (tile >= lb.num_tiles) return;
    const int64_t l0 = (int64_t)tile * MJ_TILE;
    const int rows = (int)min((int64_t)MJ_TILE, nl - l0);
    uint32_t c[MJ_ITEMS], sum = 0;
    // the warp's left rows are l0 + 128 w .. + 127: bracket their right ranges
    const int wf = (int)warp * 32 * MJ_ITEMS;
    int64_t a0 = 0, b0 = nr;
    if (wf < rows) warp_bracket(RK, LK, nk, nr, l0 + wf, l0 + min(wf + 32 * MJ_ITEMS, rows) - 1, &a0, &b0);
#pragma unroll
    for (int i = 0; i < MJ_ITEMS; ++i) {  // thread t: left rows l0 + 4t .. 4t + 3
        const int li = (int)threadIdx.x * MJ_ITEMS + i;
        const int64_t l = l0 + li;
        uint32_t cnt = 0, lo = 0;
        if (li < rows) {
            if (!has_zero(LK, l, nk)) {
                int64_t a, a2;
                eq_range(RK, LK, l, nk, a0, b0, &a, &a2);
                lo = (uint32_t)a;
                cnt = (uint32_t)(a2 - a);
            }
            if (left && cnt == 0) {
                cnt = 1;
                lo = NO_MATCH;
            }
            s_lo[li] = lo;
        }
        c[i] = cnt;
        sum += cnt;
    }
    uint32_t x = sum;  // block exclusive scan of the per-thread sums
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((int)lane >= d) x += y;
    }
    if (lane == 31) s_wsum[warp] = x;
    __syncthreads();
    uint32_t wb = 0, tot = 0;
    for (int w = 0; w < MJ_THREADS / 32; ++w) {
        if (w < (int)warp) wb += s_wsum[w];
        tot += s_wsum[w];
    }
    uint32_t run = wb + x - sum;
#pragma unroll
    for (int i = 0; i < MJ_ITEMS; ++i) {
        s_excl[threadIdx.x * MJ_ITEMS + i] = run;
        run += c[i];
    }
    if (threadIdx.x == 0) s_excl[MJ_TILE] = tot;
    if (warp == 0) {
        const long long excl = lb_exclusive_prefix(lb, tile, tot);
        if (lane == 0) {
            s_prefix = excl;
            if (tile == lb.num_tiles - 1 && excl >= 0) {
                *d_rows = excl + tot;
                *h_rows = excl + tot;
            }
        }
    }
    __syncthreads();
    const long long base = s_prefix;
    if (base < 0) return;
    for (uint32_t o = threadIdx.x; o < tot; o += MJ_THREADS) {
        int a = 0, b = rows;  // first local row whose exclusive count exceeds o
        while (a < b) {
            const int m = (a + b) >> 1;
            if (s_excl[m] <= o) a = m + 1;
            else b = m;
        }
        const int li = a - 1;
        const long long pos = base + o;
        if (pos >= cap) continue;
        const int64_t j = s_lo[li] == NO_MATCH ? -1 : (int64_t)s_lo[li] + (o - s_excl[li]);
        write_out(L, kl, Rrest, nrest, l0 + li, j, outL, outR, pos);
    }
}

// ---- hash ---------------------------------------------------------------------

constexpr unsigned long long EMPTY = ~0ull;
constexpr int SMEM_SLOTS = 2048;

__device__ __forceinline__ unsigned long long hash_key(const Cols &K, int64_t r, int nk) {
    unsigned long long h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        if (c < nk) {
            h ^= (unsigned long long)(uint32_t)K.c[c][r];
            h *= 0xFF51AFD7ED558CCDull;
            h ^= h >> 33;
            h *= 0xC4CEB9FE1A85EC53ull;
            h ^= h >> 29;
        }
    }
    return h;
}

__device__ __forceinline__ unsigned long long make_entry(unsigned long long h, int64_t row) {
    return ((h >> 32) << 32) | (unsigned long long)(uint32_t)row;
}

__global__ void k_hash_build(Cols BK, int64_t nb, int nk, unsigned long long *__restrict__ slots,
                             uint32_t *__restrict__ cnt, uint32_t mask, int *__restrict__ err) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        if (has_zero(BK, b, nk)) continue;
        const unsigned long long h = hash_key(BK, b, nk);
        const unsigned long long e = make_entry(h, b);
        uint32_t idx = (uint32_t)h & mask;
        bool done = false;
        for (uint32_t probe = 0; probe <= mask && !done; ++probe) {
            unsigned long long cur = slots[idx];
            if (cur == EMPTY) {
                const unsigned long long old = atomicCAS(slots + idx, EMPTY, e);
                if (old == EMPTY) {
                    atomicAdd(cnt + idx, 1u);
                    done = true;
                    break;
                }
                cur = old;
            }
            if ((cur >> 32) == (e >> 32) && cmp_rows(BK, (int64_t)(uint32_t)cur, BK, b, nk) == 0) {
                atomicAdd(cnt + idx, 1u);
                done = true;
                break;
            }
            idx = (idx + 1) & mask;
        }
        if (!done) atomicExch(err, TID_ERR_CAPACITY);
    }
}

// slot of B row b's key (its key was inserted); -1 if absent
__device__ __forceinline__ int64_t find_slot(const unsigned long long *slots, uint32_t mask, const Cols &BK,
                                             const Cols &QK, int64_t q, int nk, unsigned long long h) {
    uint32_t idx = (uint32_t)h & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long cur = slots[idx];
        if (cur == EMPTY) return -1;
        if ((cur >> 32) == (h >> 32) && cmp_rows(BK, (int64_t)(uint32_t)cur, QK, q, nk) == 0) return idx;
        idx = (idx + 1) & mask;
    }
    return -1;
}

__global__ void k_hash_scatter(Cols BK, int64_t nb, int nk, const unsigned long long *__restrict__ slots,
                               uint32_t mask, const uint32_t *__restrict__ start, uint32_t *__restrict__ cursor,
                               int32_t *__restrict__ grouped) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        if (has_zero(BK, b, nk)) continue;
        const int64_t s = find_slot(slots, mask, BK, BK, b, nk, hash_key(BK, b, nk));
        if (s < 0) continue;
        const uint32_t pos = start[s] + atomicAdd(cursor + s, 1u);
        grouped[pos] = (int32_t)b;
    }
}

template <bool SMEM>
__global__ void k_hash_count(Cols QK, int64_t nq, Cols BK, int nk, const unsigned long long *__restrict__ g_slots,
                             const uint32_t *__restrict__ g_cnt, const uint32_t *__restrict__ g_start, uint32_t mask,
                             uint32_t *__restrict__ cnt, uint32_t *__restrict__ qstart,
                             unsigned long long *__restrict__ total) {
    __shared__ unsigned long long s_slots[SMEM ? SMEM_SLOTS : 1];
    __shared__ uint32_t s_cnt[SMEM ? SMEM_SLOTS : 1], s_start[SMEM ? SMEM_SLOTS : 1];
    const unsigned long long *slots = g_slots;
    const uint32_t *scnt = g_cnt, *sstart = g_start;
    if (SMEM) {
        for (uint32_t i = threadIdx.x; i <= mask; i += blockDim.x) {
            s_slots[i] = g_slots[i];
            s_cnt[i] = g_cnt[i];
            s_start[i] = g_start[i];
        }
        __syncthreads();
        slots = s_slots;
        scnt = s_cnt;
        sstart = s_start;
    }
    // HC_U probe rows per thread per step, hashed first so that their key
    // loads are in flight together
    constexpr int HC_U = 4;
    unsigned long long acc = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * HC_U;
    for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x * HC_U + threadIdx.x; q0 < nq; q0 += stride) {
        unsigned long long h[HC_U];
        bool z[HC_U];
#pragma unroll
        for (int u = 0; u < HC_U; ++u) {
            const int64_t q = min(q0 + (int64_t)u * blockDim.x, nq - 1);
            h[u] = hash_key(QK, q, nk);
            z[u] = has_zero(QK, q, nk);
        }
#pragma unroll
        for (int u = 0; u < HC_U; ++u) {
            const int64_t q = q0 + (int64_t)u * blockDim.x;
            if (q >= nq) break;
            uint32_t c = 0, st = 0;
            if (!z[u]) {
                const int64_t s = find_slot(slots, mask, BK, QK, q, nk, h[u]);
                if (s >= 0) {
                    c = scnt[s];
                    st = sstart[s];
                }
            }
            cnt[q] = c;
            qstart[q] = st;
            acc += c;
        }
    }
    block_add_u64(acc, total);  // once per warp: one address takes these atomics one at a time
}

struct Scratch {
    tid_ctx *ctx;
    std::vector<void *> ptrs;
    explicit Scratch(tid_ctx *c) : ctx(c) {}
    ~Scratch() {
        for (void *p : ptrs) dev_free(ctx, p);
    }
    template <class T>
    int get(T **p, size_t count) {
        void *q = nullptr;
        TID_TRY(dev_alloc(ctx, &q, count * sizeof(T) + 16));
        ptrs.push_back(q);
        *p = (T *)q;
        return TID_OK;
    }
};

int read_u64(tid_ctx *ctx, const unsigned long long *d, unsigned long long *h) {
    TID_TRY_CUDA(cudaMemcpyAsync(h, d, 8, cudaMemcpyDeviceToHost, ctx->stream), "read count");
    TID_TRY_CUDA(cudaStreamSynchronize(ctx->stream), "read count");
    return check_ctx_error(ctx);
}

}  // namespace

int join_sets(tid_ctx *ctx, const tid_set *L, const tid_set *R, int algo, tid_set **out, bool sorted_out) {
    *out = nullptr;
    if (algo & TID_JOIN_RIGHT) return outer_join_sets(ctx, L, R, algo, out);
    const bool left = (algo & TID_JOIN_LEFT) != 0;
    algo &= ~TID_JOIN_LEFT;
    int64_t nl = 0, nr = 0;
    TID_TRY(set_rows_host(L, &nl));
    TID_TRY(set_rows_host(R, &nr));
    // schema: shared variables, R's other columns
    int lkey[TID_MAX_COLS], rkey[TID_MAX_COLS], rrest[TID_MAX_COLS];
    int nk = 0, nrest = 0;
    for (int c = 0; c < L->k; ++c)
        for (int d = 0; d < R->k; ++d)
            if (L->vars[c] == R->vars[d]) {
                lkey[nk] = c;
                rkey[nk] = d;
                ++nk;
            }
    for (int d = 0; d < R->k; ++d) {
        bool shared = false;
        for (int c = 0; c < L->k; ++c) shared = shared || L->vars[c] == R->vars[d];
        if (!shared) rrest[nrest++] = d;
    }
    const int kout = L->k + nrest;
    if (kout > TID_MAX_COLS) return fail(TID_ERR_ARG, "tid_join: output would have %d columns", kout);
    int8_t ovars[TID_MAX_COLS];
    for (int c = 0; c < L->k; ++c) ovars[c] = L->vars[c];
    for (int c = 0; c < nrest; ++c) ovars[L->k + c] = R->vars[rrest[c]];
    if (algo != TID_JOIN_AUTO && algo != TID_JOIN_SORT_MERGE && algo != TID_JOIN_HASH)
        return fail(TID_ERR_ARG, "tid_join: unknown algorithm %d", algo);

    if (left && algo == TID_JOIN_HASH)
        return fail(TID_ERR_ARG, "tid_join: a left outer join runs as a sort-merge join");
    if (left && nl > 0 && nr == 0) {  // every left row, unbound on the right
        tid_set *e = nullptr;
        TID_TRY(set_alloc(ctx, kout, ovars, nl, &e));
        int rc = TID_OK;
        for (int c = 0; c < kout && rc == TID_OK; ++c) {
            cudaError_t ce = c < L->k ? cudaMemcpyAsync(e->col[c], L->col[c], (size_t)nl * 4, cudaMemcpyDeviceToDevice,
                                                        ctx->stream)
                                      : cudaMemsetAsync(e->col[c], 0, (size_t)nl * 4, ctx->stream);
            if (ce != cudaSuccess) rc = fail_cuda(ce, "tid_join: left rows");
        }
        e->bounded = L->bounded;
        for (int c = 0; c < kout; ++c) {
            e->lo[c] = c < L->k ? L->lo[c] : 0x80000000u;
            e->hi[c] = c < L->k ? L->hi[c] : 0x80000000u;
        }
        if (rc == TID_OK) rc = set_rows_const(e, nl);
        if (rc == TID_OK) rc = set_ready(e);
        if (rc != TID_OK) {
            set_free(e);
            return rc;
        }
        *out = e;
        return TID_OK;
    }
    if (nl == 0 || nr == 0) {
        tid_set *e = nullptr;
        TID_TRY(set_alloc(ctx, kout, ovars, 0, &e));
        int rc = set_rows_const(e, 0);
        if (rc == TID_OK) rc = set_ready(e);
        if (rc != TID_OK) {
            set_free(e);
            return rc;
        }
        *out = e;
        return TID_OK;
    }
    bool lprefix = true, rprefix = true;
    for (int i = 0; i < nk; ++i) {
        lprefix = lprefix && lkey[i] == i;
        rprefix = rprefix && rkey[i] == i;
    }
    if (algo == TID_JOIN_AUTO) algo = (nk == 0 || (lprefix && rprefix)) ? TID_JOIN_SORT_MERGE : TID_JOIN_HASH;
    if (nk == 0 || left) algo = TID_JOIN_SORT_MERGE;  // cross product; left outer join
    if (!sorted_out && (algo != TID_JOIN_HASH || nk == 0 || left))
        return fail(TID_ERR_ARG, "join: unsorted output is for inner hash joins");

    cudaStream_t st = ctx->stream;
    Bounds b{};  // output columns keep their input's bounds
    for (int c = 0; c < L->k; ++c) {
        b.lo[c] = L->lo[c];
        b.hi[c] = L->hi[c];
    }
    for (int c = 0; c < nrest; ++c) {
        b.lo[L->k + c] = left ? std::min(R->lo[rrest[c]], 0x80000000u) : R->lo[rrest[c]];  // 0 pads
        b.hi[L->k + c] = left ? std::max(R->hi[rrest[c]], 0x80000000u) : R->hi[rrest[c]];
    }
    const bool bounded = L->bounded && R->bounded;
    auto finish = [&](tid_set *res) {
        res->bounded = bounded;
        for (int c = 0; c < kout && bounded; ++c) {
            res->lo[c] = b.lo[c];
            res->hi[c] = b.hi[c];
        }
        *out = res;
        return TID_OK;
    };
    if (sorted_out && algo == TID_JOIN_SORT_MERGE && nk > 0 && lprefix && rprefix && (L->k == nk || R->k == nk)) {
        // single pass into a result sized by the bound on its rows
        const int64_t ub = (L->k == nk ? nr : nl) + (left && L->k == nk ? nl : 0);
        tid_set *res = nullptr;
        TID_TRY(set_alloc(ctx, kout, ovars, ub, &res));
        Cols LK{}, RK{}, Lc{}, Rc{};
        for (int i = 0; i < nk; ++i) {
            LK.c[i] = L->col[i];
            RK.c[i] = R->col[i];
        }
        MCols oL{}, oR{};
        for (int c = 0; c < L->k; ++c) {
            Lc.c[c] = L->col[c];
            oL.c[c] = res->col[c];
        }
        for (int c = 0; c < nrest; ++c) {
            Rc.c[c] = R->col[rrest[c]];
            oR.c[c] = res->col[L->k + c];
        }
        const unsigned tiles = (unsigned)ceil_div(nl, (int64_t)MJ_TILE);
        Lookback lb{};
        int rc = lookback_scratch(ctx, tiles, &lb);
        if (rc == TID_OK) {
            k_merge_join<<<tiles, MJ_THREADS, 0, st>>>(LK, nl, RK, nr, nk, left, Lc, L->k, Rc, nrest, oL, oR,
                                                      res->cap, res->d_rows, res->slot.dev, lb);
            rc = launch_check("k_merge_join");
        }
        if (rc == TID_OK) rc = set_ready(res);
        if (rc != TID_OK) {
            set_free(res);
            return rc;
        }
        return finish(res);
    }
    Scratch s(ctx);
    Cols Lall{}, Rrest{};
    for (int c = 0; c < L->k; ++c) Lall.c[c] = L->col[c];
    for (int c = 0; c < nrest; ++c) Rrest.c[c] = R->col[rrest[c]];
    unsigned long long *d_total = nullptr;
    TID_TRY(s.get(&d_total, 1));
    TID_TRY_CUDA(cudaMemsetAsync(d_total, 0, 8, st), "memset");

    uint32_t *off = nullptr, *lo = nullptr;
    const int32_t *lperm = nullptr, *rperm = nullptr, *rmap = nullptr;
    int64_t n_probe = nl;
    bool left_is_probe = true;
    // The rows come out already canonical (sorted, distinct) when both inputs
    // lead with the shared variables in the same order: a sort-merge join walks
    // L in its order and each left row's matches in R's order, so the output is
    // ordered by L's columns, then by R's other columns; a hash join does the
    // same when its build side holds only the key columns (at most one match
    // per probe row, the output ordered as the probe side).  Then no output sort.
    bool canonical_out = false;

    if (algo == TID_JOIN_SORT_MERGE) {
        Cols LK{}, RK{};
        // left keys in key order
        if (lprefix) {
            for (int i = 0; i < nk; ++i) LK.c[i] = L->col[i];
        } else {
            int32_t *p = nullptr;
            TID_TRY(s.get(&p, nl));
            const int32_t *kc[TID_MAX_COLS];
            for (int i = 0; i < nk; ++i) kc[i] = L->col[lkey[i]];
            TID_TRY(sort_perm(ctx, kc, nk, nl, p));
            int32_t *g[TID_MAX_COLS];
            for (int i = 0; i < nk; ++i) TID_TRY(s.get(&g[i], nl));
            TID_TRY(gather_cols(ctx, kc, nk, p, nl, g));
            for (int i = 0; i < nk; ++i) LK.c[i] = g[i];
            lperm = p;
        }
        if (rprefix) {
            for (int i = 0; i < nk; ++i) RK.c[i] = R->col[i];
        } else {
            int32_t *p = nullptr;
            TID_TRY(s.get(&p, nr));
            const int32_t *kc[TID_MAX_COLS];
            for (int i = 0; i < nk; ++i) kc[i] = R->col[rkey[i]];
            TID_TRY(sort_perm(ctx, kc, nk, nr, p));
            int32_t *g[TID_MAX_COLS];
            for (int i = 0; i < nk; ++i) TID_TRY(s.get(&g[i], nr));
            TID_TRY(gather_cols(ctx, kc, nk, p, nr, g));
            for (int i = 0; i < nk; ++i) RK.c[i] = g[i];
            rperm = p;
        }
        uint32_t *cnt = nullptr;
        TID_TRY(s.get(&cnt, nl));
        TID_TRY(s.get(&lo, nl));
        TID_TRY(s.get(&off, nl));
        canonical_out = lprefix && rprefix;
        k_sm_count<<<grid_for(nl, 256), 256, 0, st>>>(LK, nl, RK, nr, nk, left, cnt, lo, d_total);
        TID_TRY(launch_check("k_sm_count"));
        TID_TRY(scan_exclusive_u32(ctx, cnt, off, nl, nullptr));
    } else {
        // build on the smaller side
        const bool build_left = nl < nr;
        const tid_set *B = build_left ? L : R;
        const tid_set *Q = build_left ? R : L;
        const int *bkey = build_left ? lkey : rkey;
        const int *qkey = build_left ? rkey : lkey;
        const int64_t nb = build_left ? nl : nr, nq = build_left ? nr : nl;
        Cols BK{}, QK{};
        for (int i = 0; i < nk; ++i) {
            BK.c[i] = B->col[bkey[i]];
            QK.c[i] = Q->col[qkey[i]];
        }
        uint32_t T = 64;
        while ((int64_t)T < 2 * nb) T <<= 1;
        const uint32_t mask = T - 1;
        unsigned long long *slots = nullptr;
        uint32_t *scnt = nullptr, *sstart = nullptr, *cursor = nullptr, *cnt = nullptr;
        int32_t *grouped = nullptr;
        TID_TRY(s.get(&slots, T));
        TID_TRY(s.get(&scnt, T));
        TID_TRY(s.get(&sstart, T));
        TID_TRY(s.get(&cursor, T));
        TID_TRY(s.get(&grouped, nb));
        TID_TRY_CUDA(cudaMemsetAsync(slots, 0xFF, (size_t)T * 8, st), "memset");
        TID_TRY_CUDA(cudaMemsetAsync(scnt, 0, (size_t)T * 4, st), "memset");
        TID_TRY_CUDA(cudaMemsetAsync(cursor, 0, (size_t)T * 4, st), "memset");
        k_hash_build<<<grid_for(nb, 256), 256, 0, st>>>(BK, nb, nk, slots, scnt, mask, ctx->err_dev);
        TID_TRY(launch_check("k_hash_build"));
        TID_TRY(scan_exclusive_u32(ctx, scnt, sstart, T, nullptr));
        k_hash_scatter<<<grid_for(nb, 256), 256, 0, st>>>(BK, nb, nk, slots, mask, sstart, cursor, grouped);
        TID_TRY(launch_check("k_hash_scatter"));
        TID_TRY(s.get(&cnt, nq));
        TID_TRY(s.get(&lo, nq));
        TID_TRY(s.get(&off, nq));
        if (T <= (uint32_t)SMEM_SLOTS)
            k_hash_count<true><<<grid_for(nq, 256 * 4), 256, 0, st>>>(QK, nq, BK, nk, slots, scnt, sstart, mask, cnt, lo, d_total);
        else
            k_hash_count<false><<<grid_for(nq, 256 * 4), 256, 0, st>>>(QK, nq, BK, nk, slots, scnt, sstart, mask, cnt, lo, d_total);
        TID_TRY(launch_check("k_hash_count"));
        TID_TRY(scan_exclusive_u32(ctx, cnt, off, nq, nullptr));
        rmap = grouped;
        n_probe = nq;
        left_is_probe = !build_left;
        canonical_out = (lprefix && rprefix && B->k == nk) || !sorted_out;
    }

    unsigned long long total = 0;
    TID_TRY(read_u64(ctx, d_total, &total));
    if (total > (unsigned long long)INT32_MAX)
        return fail(TID_ERR_CAPACITY, "tid_join: %llu output rows exceed 2^31-1", total);
    if (canonical_out) {  // write straight into the result set
        tid_set *res = nullptr;
        TID_TRY(set_alloc(ctx, kout, ovars, (int64_t)total, &res));
        MCols oL{}, oR{};
        for (int c = 0; c < L->k; ++c) oL.c[c] = res->col[c];
        for (int c = 0; c < nrest; ++c) oR.c[c] = res->col[L->k + c];
        int rc = TID_OK;
        if (total > 0) {
            k_join_write<<<(unsigned)ceil_div(n_probe + (int64_t)total, JW_TILE), JW_THREADS, 0, st>>>(
                off, n_probe, lo, lperm, rmap, rperm, (int64_t)total, Lall, L->k, Rrest, nrest, oL, oR, left_is_probe);
            rc = launch_check("k_join_write");
        }
        if (rc == TID_OK) rc = set_rows_const(res, (int64_t)total);
        if (rc == TID_OK) rc = set_ready(res);
        if (rc != TID_OK) {
            set_free(res);
            return rc;
        }
        return finish(res);
    }
    // write, then sort to canonical order
    MCols oc{}, oL{}, oR{};
    for (int c = 0; c < kout; ++c) TID_TRY(s.get(&oc.c[c], total > 0 ? total : 1));
    for (int c = 0; c < L->k; ++c) oL.c[c] = oc.c[c];
    for (int c = 0; c < nrest; ++c) oR.c[c] = oc.c[L->k + c];
    if (total > 0) {
        k_join_write<<<(unsigned)ceil_div(n_probe + (int64_t)total, JW_TILE), JW_THREADS, 0, st>>>(
            off, n_probe, lo, lperm, rmap, rperm, (int64_t)total, Lall, L->k, Rrest, nrest, oL, oR, left_is_probe);
        TID_TRY(launch_check("k_join_write"));
    }
    const int32_t *ocols[TID_MAX_COLS];
    for (int c = 0; c < kout; ++c) ocols[c] = oc.c[c];
    return canonicalize(ctx, ocols, kout, ovars, (int64_t)total, false, bounded ? &b : nullptr, out);
}

}  // namespace tid
