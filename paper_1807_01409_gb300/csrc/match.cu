// K1: single-pattern scan + order-preserving compaction.
//
// Section 3 / Algorithm 1 of the paper: every triple is tested against the key
// (0 = "?") by its own thread, and the matching positions are reported.  The
// paper marks a boolean positionArray and copies it back to the host; here the
// hits are compacted on the device, in ascending order, in ONE pass over the
// bound columns:
//
//  * persistent CTAs of 256 threads (grid = SMs x resident CTAs) loop over
//    tiles of 8192 (one bound column) or 4096 (two or three) consecutive
//    triples drawn from a ticket counter; each thread issues 16-byte loads
//    (streamed past L1, 256-byte L2 prefetch) for the NEXT tile before the
//    current tile's look-back and writes, so a CTA keeps 32-48 KB in flight;
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

// Load groups (16-byte loads per thread per bound column) by bound-column
// count: one column -> 8 (tile of 8192 triples), two or three -> 4 (4096).
template <int MASK>
struct K1Shape {
    static constexpr int B = ((MASK & 1) ? 1 : 0) + ((MASK & 2) ? 1 : 0) + ((MASK & 4) ? 1 : 0);
    static constexpr int G = B == 1 ? 8 : 4;
    static constexpr int TILE = K1_THREADS * 4 * G;
};

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

// four consecutive elements e0..e0+3 of a column; elements at or past n read as 0
template <bool VEC>
__device__ __forceinline__ int4 load4(const int32_t *__restrict__ c, int64_t e0, int64_t n) {
    if (VEC && e0 + 3 < n) return ld_stream_v4(c + e0);
    int4 v = make_int4(0, 0, 0, 0);
    if (e0 < n) v.x = ld_stream(c + e0);
    if (e0 + 1 < n) v.y = ld_stream(c + e0 + 1);
    if (e0 + 2 < n) v.z = ld_stream(c + e0 + 2);
    if (e0 + 3 < n) v.w = ld_stream(c + e0 + 3);
    return v;
}

__device__ __forceinline__ unsigned eq4(int4 v, int32_t k) {
    return (unsigned)(v.x == k) | ((unsigned)(v.y == k) << 1) |
           ((unsigned)(v.z == k) << 2) | ((unsigned)(v.w == k) << 3);
}

// Persistent, software-pipelined scan: each CTA loops over tiles drawn from the
// ticket counter.  The next tile's ticket is drawn and its loads are issued
// before the current tile's look-back and writes, so those latencies overlap
// the next tile's memory traffic.
template <int MASK, bool VEC>
__global__ void __launch_bounds__(K1_THREADS)
k1_match(const int32_t *__restrict__ S, const int32_t *__restrict__ P, const int32_t *__restrict__ O,
         int64_t n, int32_t ks, int32_t kp, int32_t ko, int32_t *__restrict__ out, int64_t cap,
         int64_t *__restrict__ d_rows, int64_t *__restrict__ h_rows, Lookback lb) {
    constexpr int G = K1Shape<MASK>::G;
    constexpr int TILE = K1Shape<MASK>::TILE;
    constexpr int NOFF = G * K1_WARPS;   // (group, warp) counts per tile: 32 or 64
    constexpr int PER_LANE = NOFF / 32;  // 1 or 2
    __shared__ unsigned s_next;
    __shared__ unsigned s_off[NOFF];
    __shared__ long long s_prefix;

    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) s_next = lb_ticket_persistent(lb, gridDim.x);
    __syncthreads();
    unsigned tile = s_next;
    bool dead = false;  // this CTA gave up a wait: mark its remaining tiles aborted

    int4 vs[G], vp[G], vo[G];
    auto issue = [&](unsigned t) {
        const int64_t tb = (int64_t)t * TILE;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int64_t e0 = tb + g * (K1_THREADS * 4) + threadIdx.x * 4;
            if (MASK & 1) vs[g] = load4<VEC>(S, e0, n);
            if (MASK & 2) vp[g] = load4<VEC>(P, e0, n);
            if (MASK & 4) vo[g] = load4<VEC>(O, e0, n);
        }
    };
    if (tile < lb.num_tiles) issue(tile);

    while (tile < lb.num_tiles) {
        const int64_t tile_base = (int64_t)tile * TILE;
        __syncthreads();  // every thread has read s_next / s_off / s_prefix of the last round
        if (threadIdx.x == 0) s_next = lb_ticket_persistent(lb, gridDim.x);

        unsigned m[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int64_t e0 = tile_base + g * (K1_THREADS * 4) + threadIdx.x * 4;
            unsigned mm = 0xFu;
            if (MASK & 1) mm &= eq4(vs[g], ks);
            if (MASK & 2) mm &= eq4(vp[g], kp);
            if (MASK & 4) mm &= eq4(vo[g], ko);
            if (e0 + 3 >= n) {  // ragged last tile
                const int64_t left = n - e0;
                mm &= left <= 0 ? 0u : (left >= 4 ? 0xFu : ((1u << left) - 1u));
            }
            m[g] = mm;
        }
        unsigned wpre[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
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
        const unsigned next = s_next;
        if (next < lb.num_tiles) issue(next);  // in flight during the look-back and writes

        if (warp == 0) {
            unsigned a[PER_LANE], sum = 0;
#pragma unroll
            for (int i = 0; i < PER_LANE; ++i) {
                a[i] = s_off[lane * PER_LANE + i];
                sum += a[i];
            }
            unsigned x = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
                if ((int)lane >= d) x += y;
            }
            unsigned run = x - sum;
#pragma unroll
            for (int i = 0; i < PER_LANE; ++i) {
                s_off[lane * PER_LANE + i] = run;
                run += a[i];
            }
            const unsigned total = __shfl_sync(0xffffffffu, x, 31);
            long long excl = -1;
            if (!dead) excl = lb_exclusive_prefix(lb, tile, total);
            else lb_abort(lb, tile);
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
        if (prefix < 0) {
            dead = true;
        } else {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const unsigned mm = m[g];
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
        tile = next;
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

int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        cached = v;
    }
    return cached;
}

template <int MASK, bool VEC>
unsigned persistent_grid(unsigned tiles) {
    static int per_sm = 0;
    if (!per_sm) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k1_match<MASK, VEC>, K1_THREADS, 0) != cudaSuccess ||
            v <= 0)
            v = 1;
        per_sm = v;
    }
    const unsigned g = (unsigned)(per_sm * sm_count());
    return tiles < g ? tiles : g;
}

template <int MASK>
int launch_mask(bool vec, cudaStream_t st, const int32_t *S, const int32_t *P, const int32_t *O,
                int64_t n, int32_t ks, int32_t kp, int32_t ko, int32_t *out, int64_t cap,
                int64_t *d_rows, int64_t *h_rows, const Lookback &lb) {
    if (vec)
        k1_match<MASK, true><<<persistent_grid<MASK, true>(lb.num_tiles), K1_THREADS, 0, st>>>(
            S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows, lb);
    else
        k1_match<MASK, false><<<persistent_grid<MASK, false>(lb.num_tiles), K1_THREADS, 0, st>>>(
            S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows, lb);
    return TID_OK;
}

int tile_of_mask(int mask) {
    switch (mask) {
        case 1: return K1Shape<1>::TILE;
        case 2: return K1Shape<2>::TILE;
        case 4: return K1Shape<4>::TILE;
        case 3: return K1Shape<3>::TILE;
        case 5: return K1Shape<5>::TILE;
        case 6: return K1Shape<6>::TILE;
        default: return K1Shape<7>::TILE;
    }
}

}  // namespace

unsigned int match_tiles(int64_t n, int mask) { return (unsigned int)ceil_div(n, tile_of_mask(mask)); }

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
    if (lb.num_tiles != match_tiles(n, mask)) return fail(TID_ERR_ARG, "k1_match: look-back scratch sized for another tiling");
    switch (mask) {
        case 1: launch_mask<1>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 2: launch_mask<2>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 3: launch_mask<3>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 4: launch_mask<4>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 5: launch_mask<5>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        case 6: launch_mask<6>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
        default: launch_mask<7>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, lb); break;
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
    if (n > 0 && mask != 0) rc = lookback_scratch(ctx, match_tiles(n, mask), &lb);
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
