// K2: several triple patterns in one pass over the store.
//
// Section 4.1 extends the search to a key array holding the keys of all
// subqueries: every triple is compared with each key and marked with the list
// of subqueries it answers (a triple may answer several, as in the paper's
// second union example).  Here the marks become one ascending index list per
// pattern, built in the same pass, with the structure of K1:
//  * each CTA streams one contiguous chunk per segment, loading the union of
//    the patterns' bound columns once per step and testing every pattern on
//    the loaded values (latency is hidden by resident warps rather than by
//    holding a second step in registers, whose pattern loop is long); each pattern keeps a triple-ordered 1-bit-per-triple
//    bitmap in shared memory (8 lanes merge 4-bit masks with three
//    xor-shuffles), 48 KB in all when one column is loaded, 96 KB otherwise, so
//    chunks shrink as patterns are added;
//  * pattern j's chunk count is a popc over its bitmap; it has one look-back
//    chain over (segment, chunk) in store order; warp w resolves the chains of
//    patterns w and w + 8;
//  * per pattern, each warp expands a contiguous run of bitmap words, 32 at a
//    time: popc, a warp prefix sum, and each lane writes the indices of its set
//    bits.
// A launch walks all segments of the store (segment = resident CTAs x chunk).
// Bytes per launch: 4 * |union of bound columns| * n read + 4 * sum of hits written.

#include <algorithm>

#include "lookback.cuh"

namespace tid {

namespace {

constexpr int K2_THREADS = 256;
constexpr int K2_WARPS = K2_THREADS / 32;
constexpr int K2_G = 8;                          // 16-byte loads per column per thread per step
constexpr int K2_STEP = K2_THREADS * 4 * K2_G;   // 8192 triples per step (256 bitmap words)

// resident CTAs per SM the register budget is shaped for: loaded data is 32
// registers per bound column
template <int U>
constexpr int k2_min_blocks() {
    return ((U & 1) + ((U >> 1) & 1) + ((U >> 2) & 1)) == 1 ? 3 : (((U & 1) + ((U >> 1) & 1) + ((U >> 2) & 1)) == 2 ? 2 : 1);
}

template <int U>
constexpr int k2_bitmap_bytes() {
    return ((U & 1) + ((U >> 1) & 1) + ((U >> 2) & 1)) == 1 ? 48 * 1024 : 96 * 1024;
}

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
__global__ void __launch_bounds__(K2_THREADS, k2_min_blocks<U>())
k2_match_multi(const int32_t *__restrict__ S, const int32_t *__restrict__ P, const int32_t *__restrict__ O,
               int64_t n, int64_t chunk_len, int n_seg, MultiArgs args, Lookback lb) {
    // pattern j's bitmap: words [j * wpp, (j+1) * wpp); bit b of word W is triple
    // c0 + 32 W + b; step st, load group g, warp w, lanes 8k..8k+7 -> word
    // st*256 + (g*8 + w)*4 + k (as in K1)
    extern __shared__ uint32_t s_bits[];
    __shared__ unsigned s_tile;
    __shared__ unsigned s_wsum[K2_WARPS];
    __shared__ long long s_prefix[TID_MAX_MULTI];

    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned sub = lane & 7u;
    const int m = args.m;
    const unsigned G = lb.num_tiles;  // chunks per segment (= grid)
    const int wpp = (int)(chunk_len / 32);
    if (threadIdx.x == 0) s_tile = lb_ticket(lb);
    __syncthreads();
    const unsigned t = s_tile;
    if (t >= G) return;
    bool dead = false;
    int4 vs[K2_G], vp[K2_G], vo[K2_G];
    auto issue = [&](int64_t base) {
        const int64_t t0 = base + threadIdx.x * 4;
        if (VEC && base + K2_STEP <= n) {
#pragma unroll
            for (int g = 0; g < K2_G; ++g) {
                if (U & 1) vs[g] = ld_stream_v4(S + t0 + g * (K2_THREADS * 4));
                if (U & 2) vp[g] = ld_stream_v4(P + t0 + g * (K2_THREADS * 4));
                if (U & 4) vo[g] = ld_stream_v4(O + t0 + g * (K2_THREADS * 4));
            }
        } else {
#pragma unroll
            for (int g = 0; g < K2_G; ++g) {
                const int64_t e0 = t0 + g * (K2_THREADS * 4);
                if (U & 1) vs[g] = load4<VEC>(S, e0, n);
                if (U & 2) vp[g] = load4<VEC>(P, e0, n);
                if (U & 4) vo[g] = load4<VEC>(O, e0, n);
            }
        }
    };

    for (int sg = 0; sg < n_seg; ++sg) {
        const int64_t c0 = ((int64_t)sg * G + t) * chunk_len;
        const int64_t c1 = min(c0 + chunk_len, n);
        const int steps = (!dead && c1 > c0) ? (int)ceil_div(c1 - c0, K2_STEP) : 0;

        // ---- stream the chunk: the loaded columns are tested against every pattern
        if (steps > 0) issue(c0);
        for (int st = 0; st < steps; ++st) {
            const int64_t base = c0 + (int64_t)st * K2_STEP;
            unsigned valid = 0xFFFFFFFFu;  // bit 4g+e: element of load group g is inside the chunk
            if (base + K2_STEP > c1) {
                valid = 0;
#pragma unroll
                for (int g = 0; g < K2_G; ++g) {
                    const int64_t left = c1 - (base + g * (K2_THREADS * 4) + threadIdx.x * 4);
                    const unsigned vm = left <= 0 ? 0u : (left >= 4 ? 0xFu : ((1u << left) - 1u));
                    valid |= vm << (4 * g);
                }
            }
            for (int j = 0; j < m; ++j) {
                const int32_t ks = args.key[j][0], kp = args.key[j][1], ko = args.key[j][2];
                uint32_t *row = s_bits + (size_t)j * wpp + (size_t)st * K2_THREADS;
#pragma unroll
                for (int g = 0; g < K2_G; ++g) {
                    unsigned mm = (valid >> (4 * g)) & 0xFu;
                    if (U & 1) mm &= eq4w(vs[g], ks);
                    if (U & 2) mm &= eq4w(vp[g], kp);
                    if (U & 4) mm &= eq4w(vo[g], ko);
                    unsigned v = mm << (4 * sub);
                    v |= __shfl_xor_sync(0xffffffffu, v, 1);
                    v |= __shfl_xor_sync(0xffffffffu, v, 2);
                    v |= __shfl_xor_sync(0xffffffffu, v, 4);
                    if (sub == (unsigned)g) row[(g * K2_WARPS + warp) * 4 + (lane >> 3)] = v;
                }
            }
            if (st + 1 < steps) issue(base + K2_STEP);  // registers are free once all patterns are tested
        }
        __syncthreads();

        // ---- chunk offsets: chain of pattern j over (segment, chunk)
        const int nwords = steps * K2_THREADS;
        const unsigned idx = (unsigned)sg * G + t;
        for (int j = (int)warp; j < m; j += K2_WARPS) {
            const uint32_t *b = s_bits + (size_t)j * wpp;
            unsigned tot = 0;
            for (int i = (int)lane; i < nwords; i += 32) tot += __popc(b[i]);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, d);
            Lookback lj = lb;
            lj.status = lb.status + (size_t)j * n_seg * G;
            lj.num_tiles = (unsigned)n_seg * G;
            long long excl = -1;
            if (!dead) excl = lb_exclusive_prefix(lj, idx, tot);
            else lb_abort(lj, idx);
            if (lane == 0) {
                s_prefix[j] = excl;
                if (idx == lj.num_tiles - 1 && excl >= 0) {
                    *args.d_rows[j] = excl + tot;
                    *args.h_rows[j] = excl + tot;
                }
            }
        }
        __syncthreads();
        for (int j = 0; j < m; ++j) dead = dead || s_prefix[j] < 0;

        // ---- expand: per pattern, warp w owns words [w0, w1), 32 at a time
        if (!dead && steps > 0) {
            const int per = (nwords / 32 + K2_WARPS - 1) / K2_WARPS * 32;
            const int w0 = min(nwords, (int)warp * per), w1 = min(nwords, w0 + per);
            for (int j = 0; j < m; ++j) {
                const uint32_t *b = s_bits + (size_t)j * wpp;
                unsigned wt = 0;
                for (int i = w0 + (int)lane; i < w1; i += 32) wt += __popc(b[i]);
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) wt += __shfl_xor_sync(0xffffffffu, wt, d);
                __syncthreads();  // s_wsum is reused
                if (lane == 0) s_wsum[warp] = wt;
                __syncthreads();
                long long run = s_prefix[j];
                for (unsigned w = 0; w < warp; ++w) run += s_wsum[w];
                int32_t *out = args.out[j];
                const int64_t cap = args.cap[j];
                for (int i0 = w0; i0 < w1; i0 += 32) {
                    uint32_t word = b[i0 + lane];
                    const unsigned c = __popc(word);
                    unsigned x = c;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
                        if ((int)lane >= d) x += y;
                    }
                    const unsigned batch = __shfl_sync(0xffffffffu, x, 31);
                    if (batch == 0) continue;
                    long long pos = run + (x - c);
                    const int64_t wbase = c0 + (int64_t)(i0 + (int)lane) * 32;
                    while (word) {
                        const int bit = __ffs(word) - 1;
                        if ((unsigned long long)pos < (unsigned long long)cap) out[pos] = (int32_t)(wbase + bit);
                        ++pos;
                        word &= word - 1;
                    }
                    run += batch;
                }
            }
        }
        __syncthreads();  // bitmaps are rewritten by the next segment
    }
}

template <int U, bool VEC>
unsigned resident_k2() {
    static unsigned cached = 0;
    if (!cached) {
        cudaFuncSetAttribute(k2_match_multi<U, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, k2_bitmap_bytes<U>());
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k2_match_multi<U, VEC>, K2_THREADS, k2_bitmap_bytes<U>()) !=
                cudaSuccess || v <= 0)
            v = 1;
        cached = (unsigned)(v * sm_count());
    }
    return cached;
}

// chunk length for m patterns: all m bitmaps fit the instance's bitmap bytes
template <int U>
int64_t k2_chunk_len(int m) {
    const int64_t bits = (int64_t)k2_bitmap_bytes<U>() * 8 / m;
    return std::max<int64_t>(K2_STEP, bits / K2_STEP * K2_STEP);
}

template <int U, bool VEC>
int launch_u(tid_ctx *ctx, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n, const MultiArgs &a) {
    const unsigned gmax = resident_k2<U, VEC>();
    int64_t chunk = k2_chunk_len<U>(a.m);
    // fewer, longer chunks are never needed: shrink the grid for small stores
    int64_t chunks = std::min<int64_t>(gmax, ceil_div(n, chunk));
    if (chunks < (int64_t)gmax) chunk = ceil_div(ceil_div(n, chunks), K2_STEP) * K2_STEP;
    chunks = std::min<int64_t>(chunks, ceil_div(n, chunk));
    const int n_seg = (int)ceil_div(n, chunks * chunk);
    Lookback lb{};
    TID_TRY(lookback_scratch(ctx, (unsigned)(chunks * n_seg * a.m), &lb));
    lb.num_tiles = (unsigned)chunks;
    k2_match_multi<U, VEC><<<(unsigned)chunks, K2_THREADS, (size_t)(chunk / 8) * a.m, ctx->stream>>>(
        S, P, O, n, chunk, n_seg, a, lb);
    return launch_check("k2_match_multi");
}

template <int U>
int launch_vec(bool vec, tid_ctx *ctx, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n,
               const MultiArgs &a) {
    return vec ? launch_u<U, true>(ctx, S, P, O, n, a) : launch_u<U, false>(ctx, S, P, O, n, a);
}

}  // namespace

}  // namespace tid

using namespace tid;

extern "C" int tid_match_multi(tid_ctx *ctx, const tid_store *st, const tid_pattern *pats, int m, tid_set **outs) {
    clear_error();
    tid::Range nvtx_range("tid_match_multi");
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
                LbScratch none{};
                rc = launch_match(ctx->stream, st->s, st->p, st->o, n, st->aligned16, 0, 0, 0, outs[j]->col[0],
                                  outs[j]->cap, outs[j]->d_rows, outs[j]->slot.dev, none);
            }
        } else {
            const bool v = st->aligned16;
            switch (U) {
                case 1: rc = launch_vec<1>(v, ctx, st->s, st->p, st->o, n, a); break;
                case 2: rc = launch_vec<2>(v, ctx, st->s, st->p, st->o, n, a); break;
                case 3: rc = launch_vec<3>(v, ctx, st->s, st->p, st->o, n, a); break;
                case 4: rc = launch_vec<4>(v, ctx, st->s, st->p, st->o, n, a); break;
                case 5: rc = launch_vec<5>(v, ctx, st->s, st->p, st->o, n, a); break;
                case 6: rc = launch_vec<6>(v, ctx, st->s, st->p, st->o, n, a); break;
                default: rc = launch_vec<7>(v, ctx, st->s, st->p, st->o, n, a); break;
            }
        }
    }
    for (int j = 0; j < m && rc == TID_OK; ++j) rc = set_ready(outs[j]);
    if (rc != TID_OK) {
        for (int j = 0; j < m; ++j) {
            set_free(outs[j]);
            outs[j] = nullptr;
        }
    }
    return rc;
}
