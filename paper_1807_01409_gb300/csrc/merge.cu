// Union of canonical sets by merging (Section 4.1's union of subquery results,
// with Section 4.3's distinct final values).
//
// Two canonical sets whose columns keep their relative order in the union
// schema (absent variables padded with 0, which never reorders rows) are
// each sorted in the union schema, so their union is a merge followed by
// dropping adjacent duplicates -- no sort.  Merge path (Odeh, Green, Mwassi,
// Shmueli and Birk, "Merge Path - Parallel Merging Made Simple", IPDPSW 2012):
//  * k_merge_split: for every tile boundary d (a multiple of MG_TILE merged
//    rows), the number of A rows among the first d merged rows, by binary
//    search along the cross diagonal (A before B on equal rows);
//  * k_merge_unique: a CTA loads its tile's A and B rows into shared memory,
//    each thread merges 8 rows along its own diagonal, then rows equal to
//    their predecessor in merged order are dropped and the kept rows written
//    in order (ballot ranks, tile offset from the decoupled look-back).
// Bytes: every input row read once, every distinct row written once (+ the
// split search, O(tiles x log n) rows).

#include <algorithm>

#include "lookback.cuh"
#include "ops.cuh"

namespace tid {

namespace {

constexpr int MG_THREADS = 256;
constexpr int MG_WARPS = MG_THREADS / 32;
constexpr int MG_ITEMS = 8;
constexpr int MG_TILE = MG_THREADS * MG_ITEMS;  // merged rows per tile

struct PadCols {  // a set's columns in union-schema order; null = absent (reads as 0)
    const int32_t *c[TID_MAX_COLS];
};

__device__ __forceinline__ int32_t pval(const PadCols &A, int c, int64_t i) { return A.c[c] ? A.c[c][i] : 0; }

// a row of A vs a row of B: -1, 0, 1 in lexicographic int32 order (column loops
// run to TID_MAX_COLS with a guard so the pointers stay in registers)
__device__ __forceinline__ int cmp_pad(const PadCols &A, int64_t i, const PadCols &B, int64_t j, int nu) {
    int r = 0;
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        if (c < nu && r == 0) {
            const int32_t x = pval(A, c, i), y = pval(B, c, j);
            r = x == y ? 0 : (x < y ? -1 : 1);
        }
    }
    return r;
}

__global__ void k_merge_split(PadCols A, int64_t na, PadCols B, int64_t nb, int nu, int64_t tiles,
                              int64_t *__restrict__ split) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles) return;
    const int64_t d = min(t * MG_TILE, na + nb);
    int64_t lo = max((int64_t)0, d - nb), hi = min(d, na);
    while (lo < hi) {  // A[mid] precedes B[d - 1 - mid]: at least mid + 1 A rows come first
        const int64_t mid = (lo + hi) >> 1;
        if (cmp_pad(A, mid, B, d - 1 - mid, nu) <= 0) lo = mid + 1;
        else hi = mid;
    }
    split[t] = lo;
}

// shared-memory rows: column c of local row r at s_rows[c * (MG_TILE + 1) + r];
// rows [0, la) are A's, [la, la + lb) B's, row MG_TILE the tile's predecessor
__device__ __forceinline__ bool rows_equal(const int32_t *s_rows, int nu, int r1, int r2) {
    bool eq = true;
    for (int c = 0; c < nu; ++c) eq = eq && s_rows[c * (MG_TILE + 1) + r1] == s_rows[c * (MG_TILE + 1) + r2];
    return eq;
}

__device__ __forceinline__ int cmp_local(const int32_t *s_rows, int nu, int r1, int r2) {
    for (int c = 0; c < nu; ++c) {
        const int32_t x = s_rows[c * (MG_TILE + 1) + r1], y = s_rows[c * (MG_TILE + 1) + r2];
        if (x != y) return x < y ? -1 : 1;
    }
    return 0;
}

__global__ void __launch_bounds__(MG_THREADS)
k_merge_unique(PadCols A, int64_t na, PadCols B, int64_t nb, int nu, const int64_t *__restrict__ split, OutCols out,
               int64_t cap, int64_t *__restrict__ d_rows, int64_t *__restrict__ h_rows, Lookback lb) {
    extern __shared__ int32_t s_rows[];  // nu x (MG_TILE + 1)
    __shared__ uint16_t s_order[MG_TILE];
    __shared__ unsigned s_off[MG_ITEMS * MG_WARPS];
    __shared__ unsigned s_tile;
    __shared__ long long s_prefix;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = lb_ticket(lb);
    __syncthreads();
    const unsigned tile = s_tile;
    if (tile >= lb.num_tiles) return;
    const int64_t d0 = (int64_t)tile * MG_TILE;
    const int64_t d1 = min(d0 + MG_TILE, na + nb);
    const int64_t a0 = split[tile], a1 = split[tile + 1];
    const int64_t b0 = d0 - a0, b1 = d1 - a1;
    const int la = (int)(a1 - a0), lb_ = (int)(b1 - b0), len = la + lb_;
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        if (c >= nu) continue;
        int32_t *col = s_rows + c * (MG_TILE + 1);
        for (int r = threadIdx.x; r < len; r += MG_THREADS)
            col[r] = r < la ? pval(A, c, a0 + r) : pval(B, c, b0 + (r - la));
    }
    // the merged row before the tile: the later (larger) of A[a0 - 1] and B[b0 - 1]
    if (threadIdx.x == 0 && d0 > 0) {
        const bool from_b = a0 == 0 || (b0 > 0 && cmp_pad(A, a0 - 1, B, b0 - 1, nu) <= 0);
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < nu) s_rows[c * (MG_TILE + 1) + MG_TILE] = from_b ? pval(B, c, b0 - 1) : pval(A, c, a0 - 1);
    }
    __syncthreads();
    // this thread's diagonal: local merged rows [dt, dt + 8)
    const int dt = min((int)threadIdx.x * MG_ITEMS, len);
    int lo = max(0, dt - lb_), hi = min(dt, la);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cmp_local(s_rows, nu, mid, la + dt - 1 - mid) <= 0) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = dt - lo;  // next A row, next B row (local)
    for (int e = 0; e < MG_ITEMS && dt + e < len; ++e) {
        const bool take_a = j >= lb_ || (i < la && cmp_local(s_rows, nu, i, la + j) <= 0);
        s_order[dt + e] = (uint16_t)(take_a ? i++ : la + j++);
    }
    __syncthreads();
    // striped: drop a row equal to its predecessor in merged order
    const unsigned lt = (1u << lane) - 1u;
    unsigned keep = 0, wpre[MG_ITEMS];
#pragma unroll
    for (int q = 0; q < MG_ITEMS; ++q) {
        const int p = q * MG_THREADS + threadIdx.x;
        bool kp = false;
        if (p < len) {
            const int prev = p > 0 ? s_order[p - 1] : MG_TILE;
            kp = (d0 + p == 0) || !rows_equal(s_rows, nu, s_order[p], prev);
        }
        keep |= (unsigned)kp << q;
        const unsigned b = __ballot_sync(0xffffffffu, kp);
        wpre[q] = __popc(b & lt);
        if (lane == 0) s_off[q * MG_WARPS + warp] = __popc(b);
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned x0 = s_off[2 * lane], x1 = s_off[2 * lane + 1];
        unsigned x = x0 + x1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += y;
        }
        const unsigned ex = x - x0 - x1;
        s_off[2 * lane] = ex;
        s_off[2 * lane + 1] = ex + x0;
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
#pragma unroll
    for (int q = 0; q < MG_ITEMS; ++q) {
        if (!((keep >> q) & 1u)) continue;
        const int p = q * MG_THREADS + threadIdx.x;
        const long long pos = prefix + s_off[q * MG_WARPS + warp] + wpre[q];
        if (pos >= cap) continue;
        const int r = s_order[p];
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c)
            if (c < nu) out.col[c][pos] = s_rows[c * (MG_TILE + 1) + r];
    }
}

struct Scratch {
    tid_ctx *ctx;
    void *p = nullptr;
    explicit Scratch(tid_ctx *c) : ctx(c) {}
    ~Scratch() {
        if (p) dev_free(ctx, p);
    }
};

}  // namespace

int merge_unique(tid_ctx *ctx, const int32_t *const *acols, int64_t na, const int32_t *const *bcols, int64_t nb,
                 int nu, tid_set *out) {
    if (nu < 1 || nu > TID_MAX_COLS) return fail(TID_ERR_ARG, "merge: %d columns", nu);
    cudaStream_t st = ctx->stream;
    if (na + nb == 0) return set_rows_const(out, 0);
    PadCols A{}, B{};
    for (int c = 0; c < nu; ++c) {
        A.c[c] = acols[c];
        B.c[c] = bcols[c];
    }
    OutCols oc{};
    for (int c = 0; c < nu; ++c) oc.col[c] = out->col[c];
    const int64_t tiles = ceil_div(na + nb, (int64_t)MG_TILE);
    Scratch s(ctx);
    TID_TRY(dev_alloc(ctx, &s.p, sizeof(int64_t) * (tiles + 1)));
    int64_t *split = (int64_t *)s.p;
    k_merge_split<<<(unsigned)ceil_div(tiles + 1, 256), 256, 0, st>>>(A, na, B, nb, nu, tiles, split);
    TID_TRY(launch_check("k_merge_split"));
    const size_t smem = sizeof(int32_t) * nu * (MG_TILE + 1);
    static bool opted = false;
    if (!opted) {
        TID_TRY_CUDA(cudaFuncSetAttribute(k_merge_unique, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sizeof(int32_t) * TID_MAX_COLS * (MG_TILE + 1))),
                     "k_merge_unique smem");
        opted = true;
    }
    Lookback lb{};
    TID_TRY(lookback_scratch(ctx, (unsigned)tiles, &lb));
    k_merge_unique<<<(unsigned)tiles, MG_THREADS, smem, st>>>(A, na, B, nb, nu, split, oc, out->cap, out->d_rows,
                                                              out->slot.dev, lb);
    return launch_check("k_merge_unique");
}

}  // namespace tid
