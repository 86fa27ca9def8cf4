// K1: single-pattern scan + order-preserving compaction.
//
// Section 3 / Algorithm 1 of the paper: every triple is tested against the key
// (0 = "?") by its own thread, and the matching positions are reported.  The
// paper marks a boolean positionArray and copies it back to the host; here the
// hits are compacted on the device, in ascending order, reading the bound
// columns once and writing each index once.  Only the columns a pattern binds
// are read (template on the bound mask).
//
// k1_scan (tid_match): one cooperative launch in three phases, so that SMs that
// stream faster also do more of the work.
//  * phase A: warps draw runs of 12 1024-triple steps from one counter (the
//    next run is drawn while the current one loads) and load them with 16-byte
//    streaming
//    loads, and write the step's 32-word hit bitmap (eight lanes merge their
//    4-bit masks with three xor-shuffles) and its hit count to global memory;
//    each step's count is also added (atomically) to the total of the CTA
//    whose fixed range of steps holds it;
//  * grid barrier; phase C: CTA c's offset is the sum of the totals of CTAs
//    before it; it scans its steps' counts in shared memory and expands each
//    step: a warp turns the step's 32 words into indices in a shared-memory
//    stage (popc, warp prefix sum, set bits) and copies the stage out with
//    coalesced stores.
// Barrier waits are bounded (LB_SPIN_LIMIT polls, then TID_ERR_TIMEOUT).
//
// k1_match (tid_match_noalloc, whose scratch is a fixed array): every CTA owns
// one contiguous chunk, streams it into a shared-memory bitmap, takes its
// output offset from one decoupled look-back over the chunk counts
// (lookback.cuh) and expands the bitmap; stores larger than (resident CTAs x
// chunk) triples take several launches.
//
// Bytes per launch: 4 * (bound columns) * n read + 4 * hits written
// (k1_scan: + n/8 bitmap written and read + 8 bytes per 1024 triples of counts).

#include <algorithm>

#include "lookback.cuh"

namespace tid {

namespace {

constexpr int K1_THREADS = 256;
constexpr int K1_WARPS = K1_THREADS / 32;
constexpr int K1_G = 8;                                   // 16-byte loads per column per thread per step
constexpr int K1_STEP = K1_THREADS * 4 * K1_G;            // 8192 triples per step
// Shared-memory hit bitmap per CTA: 48 KB (384K triples) when one column is
// bound, so four CTAs fit an SM (registers allow four); 96 KB (768K triples)
// for two or three columns, whose register use allows two CTAs per SM.  Either
// way a 200M-triple store is one launch.
template <int MASK>
constexpr int k1_bitmap_bytes() {
    return ((MASK & 1) + ((MASK >> 1) & 1) + ((MASK >> 2) & 1)) == 1 ? 48 * 1024 : 96 * 1024;
}

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

template <int MASK, bool VEC>
__global__ void __launch_bounds__(K1_THREADS)
k1_match(const int32_t *__restrict__ S, const int32_t *__restrict__ P, const int32_t *__restrict__ O,
         int64_t n, int64_t seg_begin, int64_t seg_end, int64_t chunk_len, int first_seg,
         int32_t ks, int32_t kp, int32_t ko, int32_t *__restrict__ out, int64_t cap,
         int64_t *__restrict__ d_rows, int64_t *__restrict__ h_rows, Lookback lb) {
    // Linear hit bitmap: bit b of word W is triple c0 + 32 W + b.  A step covers
    // 8192 triples = 256 words; thread (warp w, lane 8k+i) loads, in load group
    // g, triples c0 + st*8192 + g*1024 + w*128 + 32k + 4i + (0..3), so the eight
    // lanes 8k..8k+7 together hold word ((st*8 + g)*8 + w)*4 + k.
    static_assert(K1_G == 8 && K1_STEP == 8192, "bitmap layout assumes 8 load groups per step");
    extern __shared__ uint32_t s_bits[];
    __shared__ unsigned s_tile;
    __shared__ unsigned s_wtot[K1_WARPS];
    __shared__ long long s_base, s_prefix;

    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_tile = lb_ticket(lb);
        s_base = first_seg ? 0 : *d_rows;  // hits of the earlier segments
    }
    __syncthreads();
    const unsigned tile = s_tile;
    if (tile >= lb.num_tiles) return;
    // an earlier segment gave up (its count stayed -1): keep -1, write nothing
    if (s_base < 0) return;
    const int64_t c0 = seg_begin + (int64_t)tile * chunk_len;
    const int64_t c1 = min(c0 + chunk_len, seg_end);
    const int steps = (int)ceil_div(c1 - c0, K1_STEP);

    // ---- phase 1: stream the chunk into the shared-memory bitmap
    int4 vs[K1_G], vp[K1_G], vo[K1_G];
    auto issue = [&](int64_t base) {
        const int64_t t0 = base + threadIdx.x * 4;
        if (VEC && base + K1_STEP <= n) {  // whole step in bounds: no per-load checks
#pragma unroll
            for (int g = 0; g < K1_G; ++g) {
                if (MASK & 1) vs[g] = ld_stream_v4(S + t0 + g * (K1_THREADS * 4));
                if (MASK & 2) vp[g] = ld_stream_v4(P + t0 + g * (K1_THREADS * 4));
                if (MASK & 4) vo[g] = ld_stream_v4(O + t0 + g * (K1_THREADS * 4));
            }
        } else {
#pragma unroll
            for (int g = 0; g < K1_G; ++g) {
                const int64_t e0 = t0 + g * (K1_THREADS * 4);
                if (MASK & 1) vs[g] = load4<VEC>(S, e0, n);
                if (MASK & 2) vp[g] = load4<VEC>(P, e0, n);
                if (MASK & 4) vo[g] = load4<VEC>(O, e0, n);
            }
        }
    };
    const unsigned sub = lane & 7u;  // position of this lane's 4 triples in its word
    unsigned cnt = 0;                 // hits recorded by this lane
    issue(c0);
    for (int st = 0; st < steps; ++st) {
        const int64_t base = c0 + (int64_t)st * K1_STEP;
        unsigned m[K1_G];
#pragma unroll
        for (int g = 0; g < K1_G; ++g) {
            unsigned mm = 0xFu;
            if (MASK & 1) mm &= eq4(vs[g], ks);
            if (MASK & 2) mm &= eq4(vp[g], kp);
            if (MASK & 4) mm &= eq4(vo[g], ko);
            m[g] = mm;
        }
        if (base + K1_STEP > c1) {  // ragged last step of the chunk
#pragma unroll
            for (int g = 0; g < K1_G; ++g) {
                const int64_t left = c1 - (base + g * (K1_THREADS * 4) + threadIdx.x * 4);
                m[g] &= left <= 0 ? 0u : (left >= 4 ? 0xFu : ((1u << left) - 1u));
            }
        }
        if (st + 1 < steps) issue(base + K1_STEP);
        uint32_t *row = s_bits + (size_t)st * (K1_THREADS);
#pragma unroll
        for (int g = 0; g < K1_G; ++g) {
            unsigned v = m[g] << (4 * sub);
            v |= __shfl_xor_sync(0xffffffffu, v, 1);
            v |= __shfl_xor_sync(0xffffffffu, v, 2);
            v |= __shfl_xor_sync(0xffffffffu, v, 4);
            if (sub == (unsigned)g) {
                row[(g * K1_WARPS + warp) * 4 + (lane >> 3)] = v;
                cnt += __popc(v);
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    if (lane == 0) s_wtot[warp] = cnt;
    __syncthreads();

    // ---- chunk offset: one look-back over the chunk counts
    if (warp == 0) {
        unsigned t = lane < K1_WARPS ? s_wtot[lane] : 0u;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
        const long long excl = lb_exclusive_prefix(lb, tile, t);
        if (lane == 0) {
            s_prefix = excl;
            if (tile == lb.num_tiles - 1 && excl >= 0) {
                *d_rows = s_base + excl + t;
                *h_rows = s_base + excl + t;
            }
        }
    }
    __syncthreads();
    if (s_prefix < 0) return;

    // ---- phase 2: expand the bitmap; warp w owns words [w0, w1), 32 at a time
    const int nwords = steps * K1_THREADS;
    const int per = (nwords / 32 + K1_WARPS - 1) / K1_WARPS * 32;
    const int w0 = min(nwords, (int)warp * per), w1 = min(nwords, w0 + per);
    unsigned wt = 0;
    for (int i = w0 + (int)lane; i < w1; i += 32) wt += __popc(s_bits[i]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) wt += __shfl_xor_sync(0xffffffffu, wt, d);
    __syncthreads();  // s_wtot is reused
    if (lane == 0) s_wtot[warp] = wt;
    __syncthreads();
    long long run = s_base + s_prefix;
    for (unsigned w = 0; w < warp; ++w) run += s_wtot[w];
    for (int i0 = w0; i0 < w1; i0 += 32) {
        uint32_t word = s_bits[i0 + lane];  // w1 - w0 is a multiple of 32
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
            const int b = __ffs(word) - 1;
            // unsigned compare: also rejects a negative base left by a segment that gave up
            if ((unsigned long long)pos < (unsigned long long)cap) out[pos] = (int32_t)(wbase + b);
            ++pos;
            word &= word - 1;
        }
        run += batch;
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

// resident CTAs of one k1 instance (opts the kernel into 64 KB of dynamic shared memory)
template <int MASK, bool VEC>
unsigned resident_ctas() {
    static unsigned cached = 0;
    if (!cached) {
        cudaFuncSetAttribute(k1_match<MASK, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, k1_bitmap_bytes<MASK>());
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k1_match<MASK, VEC>, K1_THREADS, k1_bitmap_bytes<MASK>()) !=
                cudaSuccess || v <= 0)
            v = 1;
        cached = (unsigned)(v * sm_count());
    }
    return cached;
}

template <int MASK, bool VEC>
int run_segments(cudaStream_t st, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n,
                 int32_t ks, int32_t kp, int32_t ko, int32_t *out, int64_t cap, int64_t *d_rows,
                 int64_t *h_rows, const LbScratch &sc) {
    const unsigned grid_max = resident_ctas<MASK, VEC>();
    const int64_t seg_max = (int64_t)grid_max * ((int64_t)k1_bitmap_bytes<MASK>() * 8);
    for (int64_t sb = 0; sb < n; sb += seg_max) {
        const int64_t len = std::min<int64_t>(n - sb, seg_max);
        int64_t chunks = std::min<int64_t>(grid_max, ceil_div(len, K1_STEP));
        const int64_t chunk_len = ceil_div(ceil_div(len, chunks), K1_STEP) * K1_STEP;
        chunks = ceil_div(len, chunk_len);
        Lookback lb{};
        TID_TRY(make_lookback(sc, (unsigned)chunks, &lb));
        k1_match<MASK, VEC><<<(unsigned)chunks, K1_THREADS, (size_t)(chunk_len / 8), st>>>(
            S, P, O, n, sb, sb + len, chunk_len, sb == 0, ks, kp, ko, out, cap, d_rows, h_rows, lb);
        TID_TRY(launch_check("k1_match"));
    }
    return TID_OK;
}

template <int MASK>
int run_mask(bool vec, cudaStream_t st, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n,
             int32_t ks, int32_t kp, int32_t ko, int32_t *out, int64_t cap, int64_t *d_rows, int64_t *h_rows,
             const LbScratch &sc) {
    return vec ? run_segments<MASK, true>(st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows, sc)
               : run_segments<MASK, false>(st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows, sc);
}

// ---- k1_scan: dynamic steps, grid barriers, ordered expansion -------------------

constexpr int K2S_STEP = 1024;                 // triples per warp step (32 lanes x 8 groups x 4)
constexpr int K2S_WORDS = K2S_STEP / 32;       // bitmap words per step
constexpr int K2S_CHUNK = K1_THREADS;          // steps scanned per round of phase C
// Steps per draw: long enough that one counter serves all warps and the warps
// stream one region of the store at a time (HBM pages), short enough that the
// last draws end together (measured on GB300: 12 best among 1-48; 64 separate
// counters over store partitions were slower).
constexpr int K2S_DRAW = 12;
constexpr int K2S_TICKET = 32;                 // step counter (own cache line in the control words)
constexpr size_t K2S_CTL_BYTES = 256;

struct ScanScratch {
    uint32_t *bits;      // K2S_WORDS words per step
    uint32_t *cnt;       // hits per step
    unsigned *ctl;       // [1] grid barrier, [K2S_TICKET] step counter
    unsigned *cta_tot;   // hits per CTA range (zeroed with the control words)
    int *err;
    int64_t steps;
};

template <int MASK, bool VEC>
__global__ void __launch_bounds__(K1_THREADS)
k1_scan(const int32_t *__restrict__ S, const int32_t *__restrict__ P, const int32_t *__restrict__ O, int64_t n,
        int32_t ks, int32_t kp, int32_t ko, int32_t *__restrict__ out, int64_t cap, int64_t *__restrict__ d_rows,
        int64_t *__restrict__ h_rows, ScanScratch sc) {
    // step j covers triples [1024 j, 1024 j + 1024); lane l loads, in group g,
    // triples 1024 j + 128 g + 4 l + (0..3), so lanes 8k..8k+7 hold word 4 g + k
    static_assert(K1_G == 8, "bitmap layout assumes 8 load groups per step");
    __shared__ uint32_t s_stage[K1_WARPS][K2S_STEP];
    __shared__ uint32_t s_cnt[K2S_CHUNK], s_off[K2S_CHUNK];
    __shared__ unsigned s_red[K1_WARPS];
    __shared__ long long s_base;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned sub = lane & 7u;

    // CTA c owns steps [c per, (c + 1) per) in phase C
    const int64_t per = (sc.steps + gridDim.x - 1) / gridDim.x;

    // ---- phase A: runs of K2S_DRAW steps drawn from one counter
    {
        unsigned *ticket = sc.ctl + K2S_TICKET;
        unsigned t = 0;  // first step of the current run
        if (lane == 0) t = atomicAdd(ticket, (unsigned)K2S_DRAW);
        t = __shfl_sync(0xffffffffu, t, 0);
        unsigned k = 0;  // position in the run
        while ((int64_t)(t + k) < sc.steps) {
            const int64_t step = (int64_t)t + k;
            unsigned nxt = 0;  // the next run, drawn while the last step of this one loads
            if (lane == 0 && k + 1 == (unsigned)K2S_DRAW) nxt = atomicAdd(ticket, (unsigned)K2S_DRAW);
            const int64_t base = step * K2S_STEP + lane * 4;
            int4 vs[K1_G], vp[K1_G], vo[K1_G];
            if (VEC && (step + 1) * K2S_STEP <= n) {
#pragma unroll
                for (int g = 0; g < K1_G; ++g) {
                    if (MASK & 1) vs[g] = ld_stream_v4(S + base + g * 128);
                    if (MASK & 2) vp[g] = ld_stream_v4(P + base + g * 128);
                    if (MASK & 4) vo[g] = ld_stream_v4(O + base + g * 128);
                }
            } else {  // ragged last step (elements past n read as 0, which no bound key equals)
#pragma unroll
                for (int g = 0; g < K1_G; ++g) {
                    if (MASK & 1) vs[g] = load4<VEC>(S, base + g * 128, n);
                    if (MASK & 2) vp[g] = load4<VEC>(P, base + g * 128, n);
                    if (MASK & 4) vo[g] = load4<VEC>(O, base + g * 128, n);
                }
            }
            unsigned c = 0;
            uint32_t *bw = sc.bits + (size_t)step * K2S_WORDS;
#pragma unroll
            for (int g = 0; g < K1_G; ++g) {
                unsigned mm = 0xFu;
                if (MASK & 1) mm &= eq4(vs[g], ks);
                if (MASK & 2) mm &= eq4(vp[g], kp);
                if (MASK & 4) mm &= eq4(vo[g], ko);
                unsigned v = mm << (4 * sub);
                v |= __shfl_xor_sync(0xffffffffu, v, 1);
                v |= __shfl_xor_sync(0xffffffffu, v, 2);
                v |= __shfl_xor_sync(0xffffffffu, v, 4);
                if (sub == (unsigned)g) {
                    __stcg(bw + g * 4 + (lane >> 3), v);
                    c += __popc(v);
                }
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
            if (lane == 0) {
                __stcg(sc.cnt + step, c);
                if (c) atomicAdd(sc.cta_tot + step / per, c);  // the total of the range that owns the step
            }
            if (++k == (unsigned)K2S_DRAW) {
                t = __shfl_sync(0xffffffffu, nxt, 0);
                k = 0;
            }
        }
    }
    if (!grid_barrier(sc.ctl + 1, gridDim.x, sc.err)) return;

    const int64_t r0 = min((int64_t)blockIdx.x * per, sc.steps), r1 = min(r0 + per, sc.steps);
    const unsigned mine = __ldcg(sc.cta_tot + blockIdx.x);

    // ---- phase C: offset of this range, then ordered expansion
    unsigned long long pre = 0, all = 0;
    for (unsigned c = threadIdx.x; c < gridDim.x; c += K1_THREADS) {
        const unsigned v = __ldcg(sc.cta_tot + c);
        all += v;
        if (c < blockIdx.x) pre += v;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        pre += __shfl_xor_sync(0xffffffffu, pre, d);
        all += __shfl_xor_sync(0xffffffffu, all, d);
    }
    __shared__ unsigned long long s_pre[K1_WARPS], s_all[K1_WARPS];
    if (lane == 0) {
        s_pre[warp] = pre;
        s_all[warp] = all;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long p = 0, a = 0;
        for (int w = 0; w < K1_WARPS; ++w) {
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
    if (mine == 0) return;  // no hit in this range
    long long run = s_base;
    for (int64_t q0 = r0; q0 < r1; q0 += K2S_CHUNK) {
        // block scan of this round's step counts
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
        for (int w = 0; w < K1_WARPS; ++w) {
            if (w < (int)warp) wb += s_red[w];
            rt += s_red[w];
        }
        s_cnt[threadIdx.x] = c;
        s_off[threadIdx.x] = wb + x - c;
        __syncthreads();
        // warp w expands steps q0 + 32 w .. q0 + 32 w + 31
        uint32_t *stage = s_stage[warp];
        for (int i = 0; i < 32; ++i) {
            const int li = (int)warp * 32 + i;
            const int64_t step = q0 + li;
            if (step >= r1) break;
            const unsigned sc_n = s_cnt[li];
            if (sc_n == 0) continue;
            uint32_t word = __ldcg(sc.bits + (size_t)step * K2S_WORDS + lane);
            const unsigned pc = __popc(word);
            unsigned xo = pc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, xo, d);
                if ((int)lane >= d) xo += y;
            }
            unsigned at = xo - pc;
            const uint32_t wbase = (uint32_t)(step * K2S_STEP) + lane * 32;
            while (word) {
                const int b = __ffs(word) - 1;
                stage[at++] = wbase + (uint32_t)b;
                word &= word - 1;
            }
            __syncwarp();
            const long long o0 = run + s_off[li];
            for (unsigned e = lane; e < sc_n; e += 32) {
                const long long pos = o0 + e;
                if ((unsigned long long)pos < (unsigned long long)cap) out[pos] = (int32_t)stage[e];
            }
            __syncwarp();
        }
        run += rt;
        __syncthreads();  // s_red, s_cnt, s_off are reused
    }
}

template <int MASK, bool VEC>
int scan_grid(unsigned *grid) {
    static unsigned cached = 0;
    if (!cached) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k1_scan<MASK, VEC>, K1_THREADS, 0) != cudaSuccess ||
            v <= 0)
            return fail(TID_ERR_CUDA, "k1_scan: no resident CTA");
        cached = (unsigned)(v * sm_count());
    }
    *grid = cached;
    return TID_OK;
}

template <int MASK, bool VEC>
int run_scan(cudaStream_t st, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n, int32_t ks,
             int32_t kp, int32_t ko, int32_t *out, int64_t cap, int64_t *d_rows, int64_t *h_rows,
             const ScanScratch &sc, unsigned grid) {
    void *args[] = {(void *)&S, (void *)&P, (void *)&O, (void *)&n, (void *)&ks, (void *)&kp, (void *)&ko,
                    (void *)&out, (void *)&cap, (void *)&d_rows, (void *)&h_rows, (void *)&sc};
    TID_TRY_CUDA(cudaLaunchCooperativeKernel((const void *)k1_scan<MASK, VEC>, dim3(grid), dim3(K1_THREADS), args, 0,
                                             st),
                 "k1_scan");
    return TID_OK;
}

}  // namespace

// Status words one K1 launch needs at most (one per CTA of the largest grid).
unsigned int match_scratch_words() {
    unsigned m = 0;
    m = std::max(m, resident_ctas<1, true>());
    m = std::max(m, resident_ctas<1, false>());
    m = std::max(m, resident_ctas<3, true>());
    m = std::max(m, resident_ctas<3, false>());
    m = std::max(m, resident_ctas<7, true>());
    m = std::max(m, resident_ctas<7, false>());
    return m;
}

// Launch K1 (or the iota kernel for (?,?,?)).  The caller guarantees: n >= 0,
// cap >= 0, out holds cap int32, sc holds at least match_scratch_words()
// status words and a zero ticket, d_rows / h_rows_dev are device-visible int64.
int launch_match(cudaStream_t st, const int32_t *S, const int32_t *P, const int32_t *O,
                 int64_t n, bool aligned16, int32_t ks, int32_t kp, int32_t ko,
                 int32_t *out, int64_t cap, int64_t *d_rows, int64_t *h_rows_dev,
                 const LbScratch &sc) {
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
    if (sc.cap < match_scratch_words()) return fail(TID_ERR_ARG, "k1_match: look-back scratch too small");
    switch (mask) {
        case 1: return run_mask<1>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, sc);
        case 2: return run_mask<2>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, sc);
        case 3: return run_mask<3>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, sc);
        case 4: return run_mask<4>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, sc);
        case 5: return run_mask<5>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, sc);
        case 6: return run_mask<6>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, sc);
        default: return run_mask<7>(aligned16, st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows_dev, sc);
    }
}

// k1_scan with scratch from the context's pool (see tid_match).
template <int MASK, bool VEC>
static int scan_with_scratch(tid_ctx *ctx, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n,
                             int32_t ks, int32_t kp, int32_t ko, int32_t *out, int64_t cap, int64_t *d_rows,
                             int64_t *h_rows) {
    cudaStream_t st = ctx->stream;
    unsigned grid = 0;
    TID_TRY((scan_grid<MASK, VEC>(&grid)));
    const int64_t steps = ceil_div(n, (int64_t)K2S_STEP);
    grid = (unsigned)std::min<int64_t>(grid, std::max<int64_t>(1, steps));
    const size_t bits_b = (size_t)steps * K2S_WORDS * 4, cnt_b = ((size_t)steps * 4 + 255) / 256 * 256;
    const size_t ctl_b = K2S_CTL_BYTES, tot_b = (size_t)grid * 4;  // control words: barriers and counters
    void *blk = nullptr;
    TID_TRY(dev_alloc(ctx, &blk, bits_b + cnt_b + ctl_b + tot_b));
    ScanScratch sc{};
    sc.bits = (uint32_t *)blk;
    sc.cnt = (uint32_t *)((char *)blk + bits_b);
    sc.ctl = (unsigned *)((char *)blk + bits_b + cnt_b);
    sc.cta_tot = (unsigned *)((char *)blk + bits_b + cnt_b + ctl_b);
    sc.err = ctx->err_dev;
    sc.steps = steps;
    int rc = TID_OK;
    cudaError_t e = cudaMemsetAsync(sc.ctl, 0, ctl_b + tot_b, st);  // control words and range totals
    if (e != cudaSuccess) rc = fail_cuda(e, "k1_scan control words");
    if (rc == TID_OK) rc = run_scan<MASK, VEC>(st, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows, sc, grid);
    dev_free(ctx, blk);
    return rc;
}

int launch_scan(tid_ctx *ctx, const int32_t *S, const int32_t *P, const int32_t *O, int64_t n, bool aligned16,
                int32_t ks, int32_t kp, int32_t ko, int32_t *out, int64_t cap, int64_t *d_rows, int64_t *h_rows) {
    const int mask = (ks != 0 ? 1 : 0) | (kp != 0 ? 2 : 0) | (ko != 0 ? 4 : 0);
    if (n == 0 || mask == 0) {  // nothing to scan, or every position: no scratch needed
        LbScratch none{};
        return launch_match(ctx->stream, S, P, O, n, aligned16, ks, kp, ko, out, cap, d_rows, h_rows, none);
    }
#define K1S_CALL(M, V) scan_with_scratch<M, V>(ctx, S, P, O, n, ks, kp, ko, out, cap, d_rows, h_rows)
    switch (mask) {
        case 1: return aligned16 ? K1S_CALL(1, true) : K1S_CALL(1, false);
        case 2: return aligned16 ? K1S_CALL(2, true) : K1S_CALL(2, false);
        case 3: return aligned16 ? K1S_CALL(3, true) : K1S_CALL(3, false);
        case 4: return aligned16 ? K1S_CALL(4, true) : K1S_CALL(4, false);
        case 5: return aligned16 ? K1S_CALL(5, true) : K1S_CALL(5, false);
        case 6: return aligned16 ? K1S_CALL(6, true) : K1S_CALL(6, false);
        default: return aligned16 ? K1S_CALL(7, true) : K1S_CALL(7, false);
    }
#undef K1S_CALL
}

}  // namespace tid

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int tid_match(tid_ctx *ctx, const tid_store *st, tid_pattern pat, tid_set **out) {
    using namespace tid;
    clear_error();
    tid::Range nvtx_range("tid_match");
    if (!ctx || !st || !out) return fail(TID_ERR_ARG, "tid_match: null argument");
    if (st->ctx != ctx) return fail(TID_ERR_ARG, "tid_match: store belongs to another context");
    if (pat.s < 0 || pat.p < 0 || pat.o < 0) return fail(TID_ERR_ID, "tid_match: negative ID in pattern");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    const int64_t n = st->n;
    const int8_t var = -1;
    tid_set *set = nullptr;
    TID_TRY(set_alloc(ctx, 1, &var, n, &set));
    int rc = launch_scan(ctx, st->s, st->p, st->o, n, st->aligned16, pat.s, pat.p, pat.o, set->col[0], set->cap,
                         set->d_rows, set->slot.dev);
    if (rc == TID_OK) rc = set_ready(set);
    if (rc != TID_OK) {
        set_free(set);
        return rc;
    }
    *out = set;
    return TID_OK;
}
