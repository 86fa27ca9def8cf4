// K4: stable LSD radix sort of tuple rows, and the canonical form of a set.
//
// The paper sorts every result vector before joining and merges the final
// results to keep distinct values (Section 4.3); it used a library mergesort.
// Here rows are ordered by sorting a permutation: for each key column from the
// last to the first, the (key, row) pairs are radix sorted stably, so the final
// permutation orders rows lexicographically.  Per column only the bits that
// vary are sorted: keys are rebased to (x - min) and the number of 8-bit digit
// passes is taken from (max - min).
//
// One digit pass = upsweep (per-tile 256-bin histogram, warp-aggregated) +
// exclusive scan of the (digit, tile) counts (look-back scan) + downsweep
// (stable in-tile rank by warp match_any, staged in shared memory so the
// scatter writes runs of equal digits contiguously).
// Bytes per pass: 4n (upsweep) + 8n read + 8n written (downsweep).

#include <algorithm>

#include "lookback.cuh"
#include "ops.cuh"

namespace tid {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 rows
constexpr int RS_BINS = 256;

struct ColPtrs {
    const int32_t *c[TID_MAX_COLS];
};
struct MutColPtrs {
    int32_t *c[TID_MAX_COLS];
};

__device__ __forceinline__ uint32_t order_key(int32_t x) { return (uint32_t)x ^ 0x80000000u; }

// per-column min and max in sort order (flipped sign bit)
__global__ void k_minmax(ColPtrs cols, int k, int64_t n, uint32_t *__restrict__ mn, uint32_t *__restrict__ mx) {
    uint32_t lo[TID_MAX_COLS], hi[TID_MAX_COLS];
    for (int c = 0; c < k; ++c) {
        lo[c] = 0xFFFFFFFFu;
        hi[c] = 0u;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < k; ++c) {
            const uint32_t v = order_key(cols.c[c][i]);
            lo[c] = min(lo[c], v);
            hi[c] = max(hi[c], v);
        }
    }
    for (int c = 0; c < k; ++c) {
        uint32_t a = lo[c], b = hi[c];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            a = min(a, __shfl_xor_sync(0xffffffffu, a, d));
            b = max(b, __shfl_xor_sync(0xffffffffu, b, d));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(mn + c, a);
            atomicMax(mx + c, b);
        }
    }
}

// keys[i] = order_key(col[src(i)]) - base, vals[i] = src(i), src = perm ? perm[i] : i
__global__ void k_prep(const int32_t *__restrict__ col, const int32_t *__restrict__ perm, int64_t n, uint32_t base,
                       uint32_t *__restrict__ keys, int32_t *__restrict__ vals) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = perm ? perm[i] : (int32_t)i;
        keys[i] = order_key(col[s]) - base;
        vals[i] = s;
    }
}

__global__ void k_iota32(int32_t *__restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)i;
}

__global__ void __launch_bounds__(RS_THREADS)
rs_upsweep(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist, uint32_t tiles) {
    __shared__ uint32_t cnt[RS_BINS];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const int64_t i = base + j * RS_THREADS + threadIdx.x;
        const bool valid = i < n;
        const unsigned d = valid ? (keys[i] >> shift) & 0xFFu : 0x100u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&cnt[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(RS_THREADS)
rs_downsweep(const uint32_t *__restrict__ kin, const int32_t *__restrict__ vin, uint32_t *__restrict__ kout,
             int32_t *__restrict__ vout, int64_t n, int shift, const uint32_t *__restrict__ offs, uint32_t tiles) {
    __shared__ uint32_t s_wcnt[RS_WARPS][RS_BINS];
    __shared__ uint32_t s_tdig[RS_BINS];
    __shared__ uint32_t s_gbase[RS_BINS];
    __shared__ uint32_t s_wsum[RS_WARPS];
    __shared__ uint32_t s_k[RS_TILE];
    __shared__ int32_t s_v[RS_TILE];

    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    const int64_t wbase = base + (int64_t)warp * (RS_ITEMS * 32);
    uint32_t k[RS_ITEMS], r[RS_ITEMS];
    int32_t v[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        const bool valid = i < n;
        k[j] = valid ? kin[i] : 0u;
        v[j] = valid ? vin[i] : 0;
    }
    // stable rank among this warp's rows with the same digit, in row order
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        const bool valid = i < n;
        const unsigned d = valid ? (k[j] >> shift) & 0xFFu : 0x100u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t b = 0;
        if (valid) b = s_wcnt[warp][d];
        __syncwarp();
        if (valid && lane == (unsigned)(__ffs(peers) - 1)) s_wcnt[warp][d] = b + __popc(peers);
        __syncwarp();
        r[j] = b + __popc(peers & lt);
    }
    __syncthreads();
    {
        const unsigned d = threadIdx.x;  // one digit per thread
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = s_wcnt[w][d];
            s_wcnt[w][d] = run;
            run += c;
        }
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < RS_WARPS ? s_wsum[lane] : 0u;
            uint32_t y = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
                if ((int)lane >= o) y += z;
            }
            if (lane < RS_WARPS) s_wsum[lane] = y - w;
        }
        __syncthreads();
        s_tdig[d] = x - run + s_wsum[warp];
        s_gbase[d] = offs[(int64_t)d * tiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        if (i < n) {
            const unsigned d = (k[j] >> shift) & 0xFFu;
            const uint32_t lp = s_tdig[d] + s_wcnt[warp][d] + r[j];
            s_k[lp] = k[j];
            s_v[lp] = v[j];
        }
    }
    __syncthreads();
    const int cnt = (int)(n - base < RS_TILE ? n - base : RS_TILE);
    for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
        const uint32_t kk = s_k[i];
        const unsigned d = (kk >> shift) & 0xFFu;
        const uint32_t gp = s_gbase[d] + ((uint32_t)i - s_tdig[d]);
        kout[gp] = kk;
        vout[gp] = s_v[i];
    }
}

__global__ void k_gather(ColPtrs in, int k, const int32_t *__restrict__ perm, int64_t n, MutColPtrs out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = perm[i];
        for (int c = 0; c < k; ++c) out.c[c][i] = in.c[c][s];
    }
}

__global__ void k_set_rows(int64_t *d_rows, int64_t *h_rows, int64_t n) {
    *d_rows = n;
    *h_rows = n;
}

unsigned grid_for(int64_t n, int threads) {
    const int64_t b = ceil_div(n, threads);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

struct Scratch {  // stream-ordered temporaries freed on scope exit
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

}  // namespace

int set_rows_const(tid_set *set, int64_t n) {
    k_set_rows<<<1, 1, 0, set->ctx->stream>>>(set->d_rows, set->slot.dev, n);
    set->rows_known = n;
    return launch_check("k_set_rows");
}

int sort_perm(tid_ctx *ctx, const int32_t *const *keys, int nk, int64_t n, int32_t *perm) {
    if (n <= 0) return TID_OK;
    if (nk < 0 || nk > TID_MAX_COLS) return fail(TID_ERR_ARG, "sort: %d key columns", nk);
    cudaStream_t st = ctx->stream;
    Scratch s(ctx);
    uint32_t *mm = nullptr;
    TID_TRY(s.get(&mm, 2 * TID_MAX_COLS));
    uint32_t hmin[TID_MAX_COLS], hmax[TID_MAX_COLS];
    if (nk > 0) {
        ColPtrs cp{};
        for (int c = 0; c < nk; ++c) cp.c[c] = keys[c];
        TID_TRY_CUDA(cudaMemsetAsync(mm, 0xFF, TID_MAX_COLS * 4, st), "memset");
        TID_TRY_CUDA(cudaMemsetAsync(mm + TID_MAX_COLS, 0, TID_MAX_COLS * 4, st), "memset");
        k_minmax<<<grid_for(n, 256), 256, 0, st>>>(cp, nk, n, mm, mm + TID_MAX_COLS);
        TID_TRY(launch_check("k_minmax"));
        uint32_t both[2 * TID_MAX_COLS];
        TID_TRY_CUDA(cudaMemcpyAsync(both, mm, sizeof both, cudaMemcpyDeviceToHost, st), "copy min/max");
        TID_TRY_CUDA(cudaStreamSynchronize(st), "sync min/max");
        for (int c = 0; c < nk; ++c) {
            hmin[c] = both[c];
            hmax[c] = both[TID_MAX_COLS + c];
        }
    }
    const unsigned tiles = (unsigned)ceil_div(n, RS_TILE);
    uint32_t *ka = nullptr, *kb = nullptr, *hist = nullptr;
    int32_t *pa = nullptr, *pb = nullptr;
    bool have_perm = false;  // pa holds the current permutation
    for (int c = nk - 1; c >= 0; --c) {
        const uint32_t range = hmax[c] - hmin[c];
        if (range == 0) continue;  // constant column: order unchanged
        int bits = 32 - __builtin_clz(range);
        const int passes = (bits + 7) / 8;
        if (!ka) {
            TID_TRY(s.get(&ka, n));
            TID_TRY(s.get(&kb, n));
            TID_TRY(s.get(&pa, n));
            TID_TRY(s.get(&pb, n));
            TID_TRY(s.get(&hist, (size_t)RS_BINS * tiles));
        }
        k_prep<<<grid_for(n, 256), 256, 0, st>>>(keys[c], have_perm ? pa : nullptr, n, hmin[c], ka, pa);
        TID_TRY(launch_check("k_prep"));
        for (int p = 0; p < passes; ++p) {
            const int shift = 8 * p;
            rs_upsweep<<<tiles, RS_THREADS, 0, st>>>(ka, n, shift, hist, tiles);
            TID_TRY(launch_check("rs_upsweep"));
            TID_TRY(scan_exclusive_u32(ctx, hist, hist, (int64_t)RS_BINS * tiles, nullptr));
            rs_downsweep<<<tiles, RS_THREADS, 0, st>>>(ka, pa, kb, pb, n, shift, hist, tiles);
            TID_TRY(launch_check("rs_downsweep"));
            std::swap(ka, kb);
            std::swap(pa, pb);
        }
        have_perm = true;
    }
    if (have_perm) {
        TID_TRY_CUDA(cudaMemcpyAsync(perm, pa, (size_t)n * 4, cudaMemcpyDeviceToDevice, st), "copy perm");
    } else {
        k_iota32<<<grid_for(n, 256), 256, 0, st>>>(perm, n);
        TID_TRY(launch_check("k_iota32"));
    }
    return TID_OK;
}

int gather_cols(tid_ctx *ctx, const int32_t *const *in, int k, const int32_t *perm, int64_t n,
                int32_t *const *out) {
    if (n <= 0) return TID_OK;
    ColPtrs ip{};
    MutColPtrs op{};
    for (int c = 0; c < k; ++c) {
        ip.c[c] = in[c];
        op.c[c] = out[c];
    }
    k_gather<<<grid_for(n, 256), 256, 0, ctx->stream>>>(ip, k, perm, n, op);
    return launch_check("k_gather");
}

int canonicalize(tid_ctx *ctx, const int32_t *const *cols, int k, const int8_t *vars, int64_t n, bool dedupe,
                 tid_set **out) {
    *out = nullptr;
    tid_set *set = nullptr;
    TID_TRY(set_alloc(ctx, k, vars, n, &set));
    int rc = TID_OK;
    if (n == 0) {
        rc = set_rows_const(set, 0);
    } else {
        int32_t *perm = nullptr;
        rc = dev_alloc(ctx, (void **)&perm, (size_t)n * 4);
        if (rc == TID_OK) rc = sort_perm(ctx, cols, k, n, perm);
        if (rc == TID_OK) {
            if (dedupe) {
                rc = compact_unique(ctx, cols, k, perm, n, set);
            } else {
                rc = gather_cols(ctx, cols, k, perm, n, set->col);
                if (rc == TID_OK) rc = set_rows_const(set, n);
            }
        }
        if (perm) dev_free(ctx, perm);
    }
    if (rc == TID_OK) rc = set_ready(set);
    if (rc != TID_OK) {
        tid_set_free(set);
        return rc;
    }
    *out = set;
    return TID_OK;
}

}  // namespace tid
