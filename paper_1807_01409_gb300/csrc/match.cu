// K1: single-pattern scan + order-preserving compaction.
//
// Section 3 / Algorithm 1 of the paper: every triple is tested against the key
// (0 = "?") by its own thread, and the matching positions are reported.  The
// paper marks a boolean positionArray and copies it back to the host; here the
// hits are compacted on the device, in ascending order, in ONE pass over the
// bound columns:
//
//  * a CTA of 256 threads owns a tile of 4096 consecutive triples; each thread
//    issues four 16-byte loads per bound column (streamed past L1, 256-byte L2
//    prefetch), so a CTA keeps 16 KB per column in flight;
//  * the hit mask is ranked inside the warp with ballots and inside the CTA
//    with a 32-entry scan of the (load group, warp) totals;
//  * the tile's output offset comes from a decoupled look-back over the tile
//    status words (lookback.cuh), so the store is read once and the index list
//    written once;
//  * only the columns a pattern binds are read (template on the bound mask).
//
// Bytes moved per launch: 4 * (bound columns) * n read + 4 * hits written.

#include "lookback.cuh"

namespace tid {

namespace {

constexpr int K1_THREADS = 256;
constexpr int K1_WARPS = K1_THREADS / 32;
constexpr int K1_GROUPS = 4;                        // 16-byte loads per thread per column
constexpr int K1_TILE = K1_THREADS * 4 * K1_GROUPS; // 4096 triples

__device__ __forceinline__ int4 ld_stream_v4(const int32_t *p) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.s32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ int32_t ld_stream(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ unsigned eq4(int4 v, int32_t k) {
    return (unsigned)(v.x == k) | ((unsigned)(v.y == k) << 1) |
           ((unsigned)(v.z == k) << 2) | ((unsigned)(v.w == k) << 3);
}

// 4-bit hit mask of elements e0..e0+3 of the bound columns (bits past n are 0)
template <int MASK, bool VEC>
__device__ __forceinline__ unsigned hits4(const int32_t *__restrict__ S, const int32_t *__restrict__ P,
                                          const int32_t *__restrict__ O, int64_t n, int64_t e0,
                                          int32_t ks, int32_t kp, int32_t ko) {
    unsigned m = 0xFu;
    if (VEC && e0 + 3 < n) {
        if (MASK & 1) m &= eq4(ld_stream_v4(S + e0), ks);
        if (MASK & 2) m &= eq4(ld_stream_v4(P + e0), kp);
        if (MASK & 4) m &= eq4(ld_stream_v4(O + e0), ko);
        return m;
    }
    m = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t i = e0 + e;
        if (i < n) {
            bool h = true;
            if (MASK & 1) h = h && ld_stream(S + i) == ks;
            if (MASK & 2) h = h && ld_stream(P + i) == kp;
            if (MASK & 4) h = h && ld_stream(O + i) == ko;
            m |= (unsigned)h << e;
        }
    }
    return m;
}

template <int MASK, bool VEC>
__global__ void __launch_bounds__(K1_THREADS)
k1_match(const int32_t *__restrict__ S, const int32_t *__restrict__ P, const int32_t *__restrict__ O,
         int64_t n, int32_t ks, int32_t kp, int32_t ko, int32_t *__restrict__ out, int64_t cap,
         int64_t *__restrict__ d_rows, int64_t *__restrict__ h_rows, Lookback lb) {
    __shared__ unsigned s_tile;
    __shared__ unsigned s_off[K1_GROUPS * K1_WARPS];  // (group, warp) exclusive offsets in tile
    __shared__ long long s_prefix;

    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = lb_ticket(lb);
    __syncthreads();
    const unsigned tile = s_tile;
    if (tile >= lb.num_tiles) return;
    const int64_t tile_base = (int64_t)tile * K1_TILE;

    unsigned m[K1_GROUPS];
    if (VEC && tile_base + K1_TILE <= n) {
        // full tile: issue every 16-byte load before the first compare
        int4 vs[K1_GROUPS], vp[K1_GROUPS], vo[K1_GROUPS];
#pragma unroll
        for (int g = 0; g < K1_GROUPS; ++g) {
            const int64_t e0 = tile_base + g * (K1_THREADS * 4) + threadIdx.x * 4;
            if (MASK & 1) vs[g] = ld_stream_v4(S + e0);
            if (MASK & 2) vp[g] = ld_stream_v4(P + e0);
            if (MASK & 4) vo[g] = ld_stream_v4(O + e0);
        }
#pragma unroll
        for (int g = 0; g < K1_GROUPS; ++g) {
            unsigned mm = 0xFu;
            if (MASK & 1) mm &= eq4(vs[g], ks);
            if (MASK & 2) mm &= eq4(vp[g], kp);
            if (MASK & 4) mm &= eq4(vo[g], ko);
            m[g] = mm;
        }
    } else {
#pragma unroll
        for (int g = 0; g < K1_GROUPS; ++g)
            m[g] = hits4<MASK, VEC>(S, P, O, n, tile_base + g * (K1_THREADS * 4) + threadIdx.x * 4, ks, kp, ko);
    }

    // rank inside the warp: hits of lower lanes in the same load group
    const unsigned lt = (1u << lane) - 1u;
    unsigned wpre[K1_GROUPS];
#pragma unroll
    for (int g = 0; g < K1_GROUPS; ++g) {
        unsigned pre = 0, tot = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const unsigned b = __ballot_sync(0xffffffffu, (m[g] >> e) & 1u);
            pre += __popc(b & lt);
            tot += __popc(b);
        }
        wpre[g] = pre;
        if (lane == 0) s_off[g * K1_WARPS + warp] = tot;
    }
    __syncthreads();

    // warp 0: scan the 32 (group, warp) totals, publish, look back
    if (warp == 0) {
        const unsigned v = s_off[lane];
        unsigned x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += y;
        }
        s_off[lane] = x - v;
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
    for (int g = 0; g < K1_GROUPS; ++g) {
        unsigned mm = m[g];
        if (!mm) continue;
        long long pos = prefix + s_off[g * K1_WARPS + warp] + wpre[g];
        const int64_t e0 = tile_base + g * (K1_THREADS * 4) + threadIdx.x * 4;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if ((mm >> e) & 1u) {
                if (pos < cap) out[pos] = (int32_t)(e0 + e);
                ++pos;
            }
        }
    }
}

// all-wildcard pattern: every position, in order
__global__ void k1_iota(int64_t n, int32_t *__restrict__ out, int64_t cap,
                        int64_t *__restrict__ d_rows, int64_t *__restrict__ h_rows) {
    const int64_t lim = n < cap ? n : cap;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < lim; i += stride) {
        if (i + 3 < lim && ((reinterpret_cast<uintptr_t>(out + i) & 15) == 0)) {
            *reinterpret_cast<int4 *>(out + i) = make_int4((int)i, (int)i + 1, (int)i + 2, (int)i + 3);
        } else {
            for (int e = 0; e < 4 && i + e < lim; ++e) out[i + e] = (int32_t)(i + e);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *d_rows = n;
        *h_rows = n;
    }
}

template <int MASK>
void launch_mask(bool vec, unsigned tiles, cudaStream_t st, const int32_t *S, const int32_t *P,
                 const int32_t *O, int64_t n, int32_t ks, int32_t kp, int32_t ko, int32_t *out,
                 int64_t cap, int64_t *d_rows, int64_t *h_rows, const Lookback &lb) {
    if (vec)
        k1_match<MASK, true><<<tiles, K1_THREADS, 0, st>>>(S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows, lb);
    else
        k1_match<MASK, false><<<tiles, K1_THREADS, 0, st>>>(S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows, lb);
}

}  // namespace

unsigned int match_tiles(int64_t n) { return (unsigned int)ceil_div(n, K1_TILE); }

// Launch K1 (or the iota kernel for (?,?,?)).  The caller guarantees: n >= 0,
// cap >= 0, out holds cap int32, lb has room for match_tiles(n) status words
// and a zero ticket, d_rows / h_rows_dev are device-visible int64 slots.
int launch_match(cudaStream_t st, const int32_t *S, const int32_t *P, const int32_t *O,
                 int64_t n, bool aligned16, int32_t ks, int32_t kp, int32_t ko,
                 int32_t *out, int64_t cap, int64_t *d_rows, int64_t *h_rows_dev,
                 const Lookback &lb) {
    const int mask = (ks != 0 ? 1 : 0) | (kp != 0 ? 2 : 0) | (ko != 0 ? 4 : 0);
    if (n == 0) {
        TID_TRY_CUDA(cudaMemsetAsync(d_rows, 0, sizeof(int64_t), st), "memset rows");
        TID_TRY_CUDA(cudaMemsetAsync(h_rows_dev, 0, sizeof(int64_t), st), "memset rows");
        return TID_OK;
    }
    if (mask == 0) {
        const int64_t work = ceil_div(n < cap ? n : cap, 4 * 256);
        const unsigned grid = (unsigned)(work < 152 * 8 ? (work > 0 ? work : 1) : 152 * 8);
        k1_iota<<<grid, 256, 0, st>>>(n, out, cap, d_rows, h_rows_dev);
        return launch_check("k1_iota");
    }
    const unsigned tiles = match_tiles(n);
    switch (mask) {
        case 1: launch_mask<1>(aligned16, tiles, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 2: launch_mask<2>(aligned16, tiles, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 3: launch_mask<3>(aligned16, tiles, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 4: launch_mask<4>(aligned16, tiles, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 5: launch_mask<5>(aligned16, tiles, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 6: launch_mask<6>(aligned16, tiles, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        default: launch_mask<7>(aligned16, tiles, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
    }
    return launch_check("k1_match");
}

}  // namespace tid

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int tid_match(tid_ctx *ctx, const tid_store *st, tid_pattern pat, tid_set **out) {
    using namespace tid;
    clear_error();
    if (!ctx || !st || !out) return fail(TID_ERR_ARG, "tid_match: null argument");
    if (st->ctx != ctx) return fail(TID_ERR_ARG, "tid_match: store belongs to another context");
    if (pat.s < 0 || pat.p < 0 || pat.o < 0) return fail(TID_ERR_ID, "tid_match: negative ID in pattern");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    const int64_t n = st->n;
    const int8_t var = -1;
    tid_set *set = nullptr;
    TID_TRY(set_alloc(ctx, 1, &var, n, &set));
    Lookback lb{};
    int rc = TID_OK;
    const int mask = (pat.s != 0) | ((pat.p != 0) << 1) | ((pat.o != 0) << 2);
    if (n > 0 && mask != 0) rc = lookback_scratch(ctx, match_tiles(n), &lb);
    if (rc == TID_OK)
        rc = launch_match(ctx->stream, st->s, st->p, st->o, n, st->aligned16, pat.s, pat.p, pat.o,
                          set->col[0], set->cap, set->d_rows, set->slot.dev, lb);
    if (rc == TID_OK) rc = set_ready(set);
    if (rc != TID_OK) {
        tid_set_free(set);
        return rc;
    }
    *out = set;
    return TID_OK;
}
