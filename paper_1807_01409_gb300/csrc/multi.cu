// K2: several triple patterns in one pass over the store.
//
// Section 4.1 extends the search to a key array holding the keys of all
// subqueries: every triple is compared with each key and marked with the list
// of subqueries it answers (a triple may answer several, as in the paper's
// second union example).  Here the marks become one ascending index list per
// pattern, built in the same pass:
//  * the union of the patterns' bound columns is loaded once per tile, with the
//    same persistent, software-pipelined loop as K1 (next tile's loads issued
//    before the current tile's look-backs and writes);
//  * each pattern has its own look-back chain (status words j*tiles..), all
//    chains share one ticket; warp w resolves the chains of patterns w, w+8;
//  * per-pattern hit masks are kept packed (16 bits per pattern); the in-warp
//    ranks are recomputed from ballots in the write phase instead of being held
//    in registers.
// Bytes per launch: 4 * |union of bound columns| * n read + 4 * sum of hits written.

#include "lookback.cuh"

namespace tid {

namespace {

constexpr int K2_THREADS = 256;
constexpr int K2_WARPS = K2_THREADS / 32;
constexpr int K2_G = 4;                           // 16-byte loads per column per thread
constexpr int K2_TILE = K2_THREADS * 4 * K2_G;    // 4096 triples
constexpr int K2_NOFF = K2_G * K2_WARPS;          // 32 (group, warp) counts per pattern

struct MultiArgs {
    int m;
    int32_t key[TID_MAX_MULTI][3];
    int32_t *out[TID_MAX_MULTI];
    int64_t cap[TID_MAX_MULTI];
    int64_t *d_rows[TID_MAX_MULTI];
    int64_t *h_rows[TID_MAX_MULTI];
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

// 4-bit mask of lanes of v equal to k, or all ones if k is "?" (0)
__device__ __forceinline__ unsigned eq4w(int4 v, int32_t k) {
    if (k == 0) return 0xFu;
    return (unsigned)(v.x == k) | ((unsigned)(v.y == k) << 1) | ((unsigned)(v.z == k) << 2) |
           ((unsigned)(v.w == k) << 3);
}

template <int U, bool VEC>
__global__ void __launch_bounds__(K2_THREADS)
k2_match_multi(const int32_t *__restrict__ S, const int32_t *__restrict__ P, const int32_t *__restrict__ O,
               int64_t n, MultiArgs args, Lookback lb) {
    __shared__ unsigned s_next;
    __shared__ unsigned s_off[TID_MAX_MULTI][K2_NOFF];
    __shared__ long long s_prefix[TID_MAX_MULTI];

    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int m = args.m;
    if (threadIdx.x == 0) s_next = lb_ticket_persistent(lb, gridDim.x);
    __syncthreads();
    unsigned tile = s_next;
    bool dead = false;

    int4 vs[K2_G], vp[K2_G], vo[K2_G];
    auto issue = [&](unsigned t) {
        const int64_t tb = (int64_t)t * K2_TILE;
#pragma unroll
        for (int g = 0; g < K2_G; ++g) {
            const int64_t e0 = tb + g * (K2_THREADS * 4) + threadIdx.x * 4;
            if (U & 1) vs[g] = load4<VEC>(S, e0, n);
            if (U & 2) vp[g] = load4<VEC>(P, e0, n);
            if (U & 4) vo[g] = load4<VEC>(O, e0, n);
        }
    };
    if (tile < lb.num_tiles) issue(tile);

    while (tile < lb.num_tiles) {
        const int64_t tile_base = (int64_t)tile * K2_TILE;
        __syncthreads();
        if (threadIdx.x == 0) s_next = lb_ticket_persistent(lb, gridDim.x);

        // valid-element mask per group (ragged last tile)
        unsigned valid = 0;
#pragma unroll
        for (int g = 0; g < K2_G; ++g) {
            const int64_t left = n - (tile_base + g * (K2_THREADS * 4) + threadIdx.x * 4);
            const unsigned vm = left <= 0 ? 0u : (left >= 4 ? 0xFu : ((1u << left) - 1u));
            valid |= vm << (4 * g);
        }
        // packed hit masks: bits 4g..4g+3 of hm[j] for load group g
        uint16_t hm[TID_MAX_MULTI];
#pragma unroll
        for (int j = 0; j < TID_MAX_MULTI; ++j) {
            unsigned bits = 0;
            if (j < m) {
#pragma unroll
                for (int g = 0; g < K2_G; ++g) {
                    unsigned mm = 0xFu;
                    if (U & 1) mm &= eq4w(vs[g], args.key[j][0]);
                    if (U & 2) mm &= eq4w(vp[g], args.key[j][1]);
                    if (U & 4) mm &= eq4w(vo[g], args.key[j][2]);
                    bits |= mm << (4 * g);
                }
                bits &= valid;
#pragma unroll
                for (int g = 0; g < K2_G; ++g) {
                    unsigned tot = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e) tot += __popc(__ballot_sync(0xffffffffu, (bits >> (4 * g + e)) & 1u));
                    if (lane == 0) s_off[j][g * K2_WARPS + warp] = tot;
                }
            }
            hm[j] = (uint16_t)bits;
        }
        __syncthreads();
        const unsigned next = s_next;
        if (next < lb.num_tiles) issue(next);

        for (int j = warp; j < m; j += K2_WARPS) {
            const unsigned v = s_off[j][lane];
            unsigned x = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
                if ((int)lane >= d) x += y;
            }
            s_off[j][lane] = x - v;
            const unsigned total = __shfl_sync(0xffffffffu, x, 31);
            Lookback lj = lb;
            lj.status = lb.status + (size_t)j * lb.num_tiles;
            long long excl = -1;
            if (!dead) excl = lb_exclusive_prefix(lj, tile, total);
            else lb_abort(lj, tile);
            if (lane == 0) {
                s_prefix[j] = excl;
                if (tile == lb.num_tiles - 1 && excl >= 0) {
                    *args.d_rows[j] = excl + total;
                    *args.h_rows[j] = excl + total;
                }
            }
        }
        __syncthreads();
        bool any_dead = false;
        for (int j = 0; j < m; ++j) any_dead = any_dead || s_prefix[j] < 0;
        if (any_dead) {
            dead = true;
        } else {
#pragma unroll
            for (int j = 0; j < TID_MAX_MULTI; ++j) {
                if (j >= m) break;
                const unsigned bits = hm[j];
                const long long prefix = s_prefix[j];
#pragma unroll
                for (int g = 0; g < K2_G; ++g) {
                    unsigned pre = 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        pre += __popc(__ballot_sync(0xffffffffu, (bits >> (4 * g + e)) & 1u) & lt);
                    const unsigned mm = (bits >> (4 * g)) & 0xFu;
                    if (!mm) continue;
                    long long pos = prefix + s_off[j][g * K2_WARPS + warp] + pre;
                    const int64_t e0 = tile_base + g * (K2_THREADS * 4) + threadIdx.x * 4;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        if ((mm >> e) & 1u) {
                            if (pos < args.cap[j]) args.out[j][pos] = (int32_t)(e0 + e);
                            ++pos;
                        }
                    }
                }
            }
        }
        tile = next;
    }
}

int sm_count_k2() {
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        cached = v;
    }
    return cached;
}

template <int U, bool VEC>
int launch_u(cudaStream_t st, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n,
             const MultiArgs &a, const Lookback &lb) {
    static int per_sm = 0;
    if (!per_sm) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k2_match_multi<U, VEC>, K2_THREADS, 0) != cudaSuccess ||
            v <= 0)
            v = 1;
        per_sm = v;
    }
    unsigned grid = (unsigned)(per_sm * sm_count_k2());
    if (grid > lb.num_tiles) grid = lb.num_tiles;
    k2_match_multi<U, VEC><<<grid, K2_THREADS, 0, st>>>(S, P, O, n, a, lb);
    return launch_check("k2_match_multi");
}

template <int U>
int launch_vec(bool vec, cudaStream_t st, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n,
               const MultiArgs &a, const Lookback &lb) {
    return vec ? launch_u<U, true>(st, S, P, O, n, a, lb) : launch_u<U, false>(st, S, P, O, n, a, lb);
}

}  // namespace

}  // namespace tid

using namespace tid;

extern "C" int tid_match_multi(tid_ctx *ctx, const tid_store *st, const tid_pattern *pats, int m, tid_set **outs) {
    clear_error();
    if (!ctx || !st || !pats || !outs) return fail(TID_ERR_ARG, "tid_match_multi: null argument");
    if (m < 1 || m > TID_MAX_MULTI) return fail(TID_ERR_ARG, "tid_match_multi: m = %d (1..%d)", m, TID_MAX_MULTI);
    if (st->ctx != ctx) return fail(TID_ERR_ARG, "tid_match_multi: store belongs to another context");
    for (int j = 0; j < m; ++j) {
        outs[j] = nullptr;
        if (pats[j].s < 0 || pats[j].p < 0 || pats[j].o < 0)
            return fail(TID_ERR_ID, "tid_match_multi: negative ID in pattern %d", j);
    }
    DeviceGuard g(ctx->device);
    const int64_t n = st->n;
    int U = 0;
    for (int j = 0; j < m; ++j) U |= (pats[j].s != 0) | ((pats[j].p != 0) << 1) | ((pats[j].o != 0) << 2);
    MultiArgs a{};
    a.m = m;
    int rc = TID_OK;
    const int8_t var = -1;
    for (int j = 0; j < m && rc == TID_OK; ++j) {
        rc = set_alloc(ctx, 1, &var, n, &outs[j]);
        if (rc != TID_OK) break;
        a.key[j][0] = pats[j].s;
        a.key[j][1] = pats[j].p;
        a.key[j][2] = pats[j].o;
        a.out[j] = outs[j]->col[0];
        a.cap[j] = outs[j]->cap;
        a.d_rows[j] = outs[j]->d_rows;
        a.h_rows[j] = outs[j]->slot.dev;
    }
    if (rc == TID_OK) {
        if (n == 0 || U == 0) {
            // nothing bound anywhere: every list is 0..n-1 (tid_match handles it)
            for (int j = 0; j < m && rc == TID_OK; ++j) {
                Lookback none{};
                rc = launch_match(ctx->stream, st->s, st->p, st->o, n, st->aligned16, 0, 0, 0, outs[j]->col[0],
                                  outs[j]->cap, outs[j]->d_rows, outs[j]->slot.dev, none);
            }
        } else {
            const unsigned tiles = (unsigned)ceil_div(n, K2_TILE);
            Lookback lb{};
            rc = lookback_scratch(ctx, tiles * (unsigned)m, &lb);
            lb.num_tiles = tiles;
            if (rc == TID_OK) {
                const bool v = st->aligned16;
                switch (U) {
                    case 1: rc = launch_vec<1>(v, ctx->stream, st->s, st->p, st->o, n, a, lb); break;
                    case 2: rc = launch_vec<2>(v, ctx->stream, st->s, st->p, st->o, n, a, lb); break;
                    case 3: rc = launch_vec<3>(v, ctx->stream, st->s, st->p, st->o, n, a, lb); break;
                    case 4: rc = launch_vec<4>(v, ctx->stream, st->s, st->p, st->o, n, a, lb); break;
                    case 5: rc = launch_vec<5>(v, ctx->stream, st->s, st->p, st->o, n, a, lb); break;
                    case 6: rc = launch_vec<6>(v, ctx->stream, st->s, st->p, st->o, n, a, lb); break;
                    default: rc = launch_vec<7>(v, ctx->stream, st->s, st->p, st->o, n, a, lb); break;
                }
            }
        }
    }
    for (int j = 0; j < m && rc == TID_OK; ++j) rc = set_ready(outs[j]);
    if (rc != TID_OK) {
        for (int j = 0; j < m; ++j) {
            tid_set_free(outs[j]);
            outs[j] = nullptr;
        }
    }
    return rc;
}
