// Batched single-pattern search: thousands of patterns in two scans of the
// store, each pattern's matches returned exactly as tid_match would (an
// ascending index list).
//
// The paper searches several subqueries in one pass through its key array
// (Section 4.1) and, for entailment, turns the distinct keys found by one search
// into a multi-key search (Section 5).  For a large batch the per-triple test
// against every key is replaced by lookups: for every bound-position mask
// present in the batch, the triple's own values under that mask form the only
// key of that mask it can answer, and one lookup in a table of the batch's
// distinct (mask, key) pairs -- "key ids" -- finds it.  The table is a
// hash-and-displace perfect hash built on the host (Belazzougui, Botelho and
// Dietzfelbinger, "Hash, displace, and compress", ESA 2009): a key's bucket
// gives a displacement, bucket and displacement give its slot, so a lookup is
// two shared-memory reads and one comparison, with no probe loop.
//
//  * pass 1 (count): warp w owns a contiguous slice of the store and counts the
//    hits of every key id in a warp-private shared-memory array (one add per
//    group of lanes that hit the same key id in a 32-triple slot, grouped with
//    match_any); the counts go to counts[w][kid];
//  * a per-key exclusive scan over the warps gives every (warp, key id) its
//    first output position, and each key id's total (one synchronisation sizes
//    all outputs exactly; the lists share one allocation);
//  * pass 2 (write): the same traversal; a hit's position is the warp's running
//    cursor for its key id plus its rank among the lanes of the slot that hit the
//    same key id, so every list is written in ascending order, without atomics
//    or a sort.
// Sub-batches of at most TID_BATCH_KEYS key ids keep table and counters in
// shared memory.
// Bytes per sub-batch: 2 x 4 * |union of bound columns| * n read + 4 * hits
// written (+ 3 x 4 * key ids * warps for counts and bases).

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "ops.cuh"

namespace tid {

namespace {

constexpr int KB_THREADS = 256;
constexpr int KB_WARPS = KB_THREADS / 32;
constexpr int KB_MAX_KIDS = TID_BATCH_KEYS;  // key ids per sub-batch
constexpr int KB_UNROLL = 8;                 // 32-triple slots loaded per iteration
constexpr int KB_FILTER_LOG = 13;            // per-column prefilter: 2^13 four-bit entries
constexpr int KB_FILTER_WORDS = (1 << KB_FILTER_LOG) / 8;

struct __align__(16) Entry {  // one table slot: key values under its mask, mask and key id
    int32_t s, p, o;
    int32_t mask_kid;  // mask in bits [30:28], key id in [27:0]; -1 = empty
};

// Hash of (mask, key under the mask), the same on host and device.  Each bound
// column's value, xor-ed with a per-column seed, goes through the 32-bit
// finaliser of MurmurHash3 (Appleby; public domain): a bijection with full
// avalanche, so the keys of a one-column mask never collide and IDs with
// arithmetic structure (values a power of two apart, entity and literal IDs
// 2^30 apart) do not line up.  The mixed values of the mask's columns are
// combined by xor, rotated per column, with a per-mask seed.  A triple's three
// mixed values are computed once and serve every mask.  Bucket and slot take
// the high bits of products (range reduction by multiply-high).
struct HashParams {
    uint32_t col[3];  // per-column seeds
    uint32_t msk[8];  // per-mask seeds
    uint32_t k4;      // slot multiplier
    uint32_t f[3];    // prefilter multipliers of s, p, o
};

inline HashParams hash_params(uint32_t seed) {
    HashParams hp;
    uint64_t z = seed;
    uint32_t v[15];
    for (int i = 0; i < 15; ++i) {  // SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        v[i] = (uint32_t)((x ^ (x >> 31)) >> 32);
    }
    for (int c = 0; c < 3; ++c) hp.col[c] = v[c];
    for (int m = 0; m < 8; ++m) hp.msk[m] = v[3 + m];
    hp.k4 = v[11] | 1u;
    for (int c = 0; c < 3; ++c) hp.f[c] = v[12 + c] | 1u;
    return hp;
}

__host__ __device__ __forceinline__ uint32_t kb_fmix(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

__host__ __device__ __forceinline__ uint32_t kb_rotl(uint32_t x, int r) { return (x << r) | (x >> (32 - r)); }

// mixed value of column c's value v
__host__ __device__ __forceinline__ uint32_t kb_colmix(const HashParams &hp, int c, uint32_t v) {
    return kb_fmix(v ^ hp.col[c]);
}

// hash of mask m from the mixed values of a triple's (or key's) columns
__host__ __device__ __forceinline__ uint32_t kb_combine(const HashParams &hp, int m, uint32_t ms, uint32_t mp,
                                                        uint32_t mo) {
    uint32_t x = hp.msk[m];
    if (m & 1) x ^= ms;
    if (m & 2) x ^= kb_rotl(mp, 11);
    if (m & 4) x ^= kb_rotl(mo, 22);
    return x;
}

__host__ __device__ __forceinline__ uint32_t kb_hash(const HashParams &hp, int m, uint32_t s, uint32_t p, uint32_t o) {
    return kb_combine(hp, m, (m & 1) ? kb_colmix(hp, 0, s) : 0u, (m & 2) ? kb_colmix(hp, 1, p) : 0u,
                      (m & 4) ? kb_colmix(hp, 2, o) : 0u);
}

// Prefilter entry of a column value (multiplicative hashing, top 13 bits).  Each
// entry holds one bit per mask that binds the column -- s: masks 1,3,5,7; p:
// 2,3,6,7; o: 4,5,6,7 -- set when some key of that mask has a value with this
// entry in the column.
__host__ __device__ __forceinline__ uint32_t kb_fentry(const HashParams &hp, int c, uint32_t v) {
    return (v * hp.f[c]) >> (32 - KB_FILTER_LOG);
}

__host__ __device__ __forceinline__ int kb_fbit(int c, int mask) {  // bit of `mask` in column c's entries
    return c == 0 ? (mask >> 1) : c == 1 ? ((mask & 1) | ((mask >> 1) & 2)) : (mask & 3);
}

// masks (bit m) a triple may answer, from its three entries (4-bit each)
__host__ __device__ __forceinline__ uint32_t kb_candidates(uint32_t es, uint32_t ep, uint32_t eo) {
    const uint32_t cs = 0x55u | ((es & 1u) << 1) | ((es & 2u) << 2) | ((es & 4u) << 3) | ((es & 8u) << 4);
    const uint32_t cp = 0x33u | ((ep & 3u) << 2) | ((ep & 12u) << 4);
    const uint32_t co = 0x0Fu | (eo << 4);
    return cs & cp & co;
}

__host__ __device__ __forceinline__ uint32_t kb_range(uint32_t x, uint32_t n) {  // floor(x * n / 2^32)
#ifdef __CUDA_ARCH__
    return __umulhi(x, n);
#else
    return (uint32_t)(((uint64_t)x * n) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint32_t kb_bucket(uint32_t h, uint32_t nb) { return kb_range(h, nb); }

__host__ __device__ __forceinline__ uint32_t kb_slot(const HashParams &hp, uint32_t h, uint32_t d, uint32_t ns) {
    return kb_range((h ^ (d * 0x9E3779B9u)) * hp.k4, ns);
}

struct BatchArgs {
    const int32_t *S, *P, *O;
    int64_t n;
    int64_t slice;           // triples per warp slice (multiple of 32 * KB_UNROLL)
    int kids;                // key ids in this sub-batch
    HashParams hp;           // hash multipliers
    uint32_t nb, ns;         // buckets, slots
    const Entry *table;      // ns slots
    const uint16_t *disp;    // nb displacements
    const uint32_t *filter;  // 3 x KB_FILTER_WORDS words (eight 4-bit entries each)
    uint32_t *counts;        // [warp][kid]: pass 1 writes counts, the scan turns them into bases
    int32_t *arena;          // the lists, list k at arena + off[k]
    const int64_t *off;
    int abs32;               // the allocation holds < 2^32 rows
};

__host__ __device__ __forceinline__ size_t kb_disp_bytes(uint32_t nb) { return (sizeof(uint16_t) * nb + 15) / 16 * 16; }

size_t kb_smem_bytes(int kids, uint32_t ns, uint32_t nb) {
    return sizeof(Entry) * ns + kb_disp_bytes(nb) + sizeof(uint32_t) * 3 * KB_FILTER_WORDS +
           sizeof(uint32_t) * KB_WARPS * kids;
}

// SKIP: a warp skips a mask's lookups when none of its lanes may answer it
// (fewer instructions when candidates are rare; a branch per mask that breaks the
// overlap of the seven lookups when they are common).  The autotuner picks it.
template <int U, bool WRITE, bool SKIP>
__global__ void __launch_bounds__(KB_THREADS) k_batch(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char kb_smem[];
    Entry *s_tab = (Entry *)kb_smem;
    uint16_t *s_disp = (uint16_t *)(s_tab + a.ns);
    uint32_t *s_filt = (uint32_t *)(kb_smem + sizeof(Entry) * a.ns + kb_disp_bytes(a.nb));
    uint32_t *s_cnt = s_filt + 3 * KB_FILTER_WORDS;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t i = threadIdx.x; i < a.ns; i += KB_THREADS) s_tab[i] = a.table[i];
    for (uint32_t i = threadIdx.x; i < a.nb; i += KB_THREADS) s_disp[i] = a.disp[i];
    for (uint32_t i = threadIdx.x; i < 3 * KB_FILTER_WORDS; i += KB_THREADS) s_filt[i] = a.filter[i];
    const int64_t gw = (int64_t)blockIdx.x * KB_WARPS + warp;
    uint32_t *cnt = s_cnt + warp * a.kids;
    uint32_t *row = a.counts + gw * a.kids;
    // pass 2 cursors: absolute positions in the lists' allocation when it holds
    // fewer than 2^32 rows (no per-hit offset load), else positions in each list
    for (int k = lane; k < a.kids; k += 32)
        cnt[k] = WRITE ? row[k] + (a.abs32 ? (uint32_t)a.off[k] : 0u) : 0u;
    __syncthreads();
    const int64_t lo = gw * a.slice, hi = min(lo + a.slice, a.n);
    for (int64_t b0 = lo; b0 < hi; b0 += 32 * KB_UNROLL) {
        int32_t vs[KB_UNROLL], vp[KB_UNROLL], vo[KB_UNROLL];
#pragma unroll
        for (int u = 0; u < KB_UNROLL; ++u) {
            const int64_t i = b0 + u * 32 + lane;
            const bool in = i < hi;
            vs[u] = (U & 1) && in ? __ldcs(a.S + i) : 0;
            vp[u] = (U & 2) && in ? __ldcs(a.P + i) : 0;
            vo[u] = (U & 4) && in ? __ldcs(a.O + i) : 0;
        }
#pragma unroll
        for (int u = 0; u < KB_UNROLL; ++u) {
            const int64_t i = b0 + u * 32 + lane;
            // masks this triple may answer (prefilter), and over the warp
            uint32_t e3[3] = {0u, 0u, 0u};
            const uint32_t v3[3] = {(uint32_t)vs[u], (uint32_t)vp[u], (uint32_t)vo[u]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!(U & (1 << c))) continue;
                const uint32_t f = kb_fentry(a.hp, c, v3[c]);
                e3[c] = (s_filt[c * KB_FILTER_WORDS + (f >> 3)] >> ((f & 7u) * 4u)) & 0xFu;
            }
            const uint32_t cand = i < hi ? kb_candidates(e3[0], e3[1], e3[2]) : 0u;
            const uint32_t any = __reduce_or_sync(0xffffffffu, cand);
            // the triple's mixed column values, shared by every mask's hash
            const uint32_t ms = (U & 1) ? kb_colmix(a.hp, 0, v3[0]) : 0u;
            const uint32_t mp = (U & 2) ? kb_colmix(a.hp, 1, v3[1]) : 0u;
            const uint32_t mo = (U & 4) ? kb_colmix(a.hp, 2, v3[2]) : 0u;
            // every candidate mask's lookup first (independent chains), then the hits
            int kid[7];
#pragma unroll
            for (int m = 1; m < 8; ++m) {
                kid[m - 1] = -1;
                if ((m & ~U) || (SKIP && !((any >> m) & 1))) continue;
                // lanes that cannot answer m read slot 0 like the others (a broadcast,
                // no extra shared-memory wavefront) and keep straight-line code
                const bool cm = (cand >> m) & 1;
                const uint32_t h = kb_combine(a.hp, m, ms, mp, mo);
                const uint32_t d = s_disp[cm ? kb_bucket(h, a.nb) : 0u];
                const Entry e = s_tab[cm ? kb_slot(a.hp, h, d, a.ns) : 0u];
                const bool hit = cm && (e.mask_kid >> 28) == m && (!(m & 1) || e.s == vs[u]) &&
                                 (!(m & 2) || e.p == vp[u]) && (!(m & 4) || e.o == vo[u]);
                kid[m - 1] = hit ? (e.mask_kid & 0x0FFFFFFF) : -1;
            }
#pragma unroll
            for (int m = 1; m < 8; ++m) {
                if ((m & ~U) || !((any >> m) & 1)) continue;
                const int k = kid[m - 1];
                if (!__any_sync(0xffffffffu, k >= 0)) continue;
                const unsigned peers = __match_any_sync(0xffffffffu, k);
                if (k >= 0) {
                    const uint32_t c = cnt[k];
                    if (WRITE) {
                        const uint32_t r = c + __popc(peers & lt);
                        a.arena[a.abs32 ? (int64_t)r : a.off[k] + r] = (int32_t)i;
                    }
                    __syncwarp(peers);
                    if (lane == (unsigned)(__ffs(peers) - 1)) cnt[k] = c + __popc(peers);
                }
                __syncwarp();
            }
        }
    }
    __syncwarp();
    if (!WRITE)
        for (int k = lane; k < a.kids; k += 32) row[k] = cnt[k];
}

// QUEUE shape: only the (triple, mask) pairs the prefilter admits are looked
// up.  For each 32-triple slot, lane l lists the masks its triple may answer;
// an exclusive scan over the lanes' counts gives each lane its place in a
// per-warp queue of (lane, mask) bytes, lane-major, so for any one mask the
// queue is in triple order.  The warp then looks the queue up 32 entries at a
// time -- an entry's triple values and mixed columns come from its lane by
// shuffle -- and counts or writes the hits as the direct shape does (lanes with
// the same key id grouped by match_any, ranked in queue order, hence in triple
// order).  Lookups per triple follow the prefilter's candidates instead of the
// number of masks present; UNROLL slots are loaded per iteration.
template <int U, bool WRITE, int UNROLL>
__global__ void __launch_bounds__(KB_THREADS) k_batch_q(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char kb_smem[];
    __shared__ uint8_t s_queue[KB_WARPS][32 * 7];
    __shared__ uint32_t s_msk[8];
    Entry *s_tab = (Entry *)kb_smem;
    uint16_t *s_disp = (uint16_t *)(s_tab + a.ns);
    uint32_t *s_filt = (uint32_t *)(kb_smem + sizeof(Entry) * a.ns + kb_disp_bytes(a.nb));
    uint32_t *s_cnt = s_filt + 3 * KB_FILTER_WORDS;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (uint32_t i = threadIdx.x; i < a.ns; i += KB_THREADS) s_tab[i] = a.table[i];
    for (uint32_t i = threadIdx.x; i < a.nb; i += KB_THREADS) s_disp[i] = a.disp[i];
    for (uint32_t i = threadIdx.x; i < 3 * KB_FILTER_WORDS; i += KB_THREADS) s_filt[i] = a.filter[i];
    if (threadIdx.x < 8) s_msk[threadIdx.x] = a.hp.msk[threadIdx.x];
    const int64_t gw = (int64_t)blockIdx.x * KB_WARPS + warp;
    uint32_t *cnt = s_cnt + warp * a.kids;
    uint32_t *row = a.counts + gw * a.kids;
    for (int k = lane; k < a.kids; k += 32)
        cnt[k] = WRITE ? row[k] + (a.abs32 ? (uint32_t)a.off[k] : 0u) : 0u;
    __syncthreads();
    uint8_t *queue = s_queue[warp];
    const int64_t lo = gw * a.slice, hi = min(lo + a.slice, a.n);
    for (int64_t b0 = lo; b0 < hi; b0 += 32 * UNROLL) {
        int32_t vs[UNROLL], vp[UNROLL], vo[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t i = b0 + u * 32 + lane;
            const bool in = i < hi;
            vs[u] = (U & 1) && in ? __ldcs(a.S + i) : 0;
            vp[u] = (U & 2) && in ? __ldcs(a.P + i) : 0;
            vo[u] = (U & 4) && in ? __ldcs(a.O + i) : 0;
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t i = b0 + u * 32 + lane;
            const uint32_t v3[3] = {(uint32_t)vs[u], (uint32_t)vp[u], (uint32_t)vo[u]};
            uint32_t e3[3] = {0u, 0u, 0u};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (!(U & (1 << c))) continue;
                const uint32_t f = kb_fentry(a.hp, c, v3[c]);
                e3[c] = (s_filt[c * KB_FILTER_WORDS + (f >> 3)] >> ((f & 7u) * 4u)) & 0xFu;
            }
            const uint32_t cand = i < hi ? kb_candidates(e3[0], e3[1], e3[2]) & 0xFEu : 0u;
            const unsigned c = __popc(cand);
            unsigned x = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
                if ((int)lane >= d) x += y;
            }
            const unsigned tot = __shfl_sync(0xffffffffu, x, 31);
            if (tot == 0) continue;
            unsigned at = x - c;
            for (uint32_t cm = cand; cm; cm &= cm - 1) queue[at++] = (uint8_t)((lane << 3) | (__ffs(cm) - 1));
            const uint32_t ms = (U & 1) ? kb_colmix(a.hp, 0, v3[0]) : 0u;
            const uint32_t mp = (U & 2) ? kb_colmix(a.hp, 1, v3[1]) : 0u;
            const uint32_t mo = (U & 4) ? kb_colmix(a.hp, 2, v3[2]) : 0u;
            __syncwarp();
            for (unsigned r0 = 0; r0 < tot; r0 += 32) {
                const unsigned e = r0 + lane;
                const unsigned qe = e < tot ? queue[e] : 0u;
                const int src = (int)(qe >> 3), m = (int)(qe & 7u);
                const int32_t ts = (U & 1) ? __shfl_sync(0xffffffffu, vs[u], src) : 0;
                const int32_t tp = (U & 2) ? __shfl_sync(0xffffffffu, vp[u], src) : 0;
                const int32_t to = (U & 4) ? __shfl_sync(0xffffffffu, vo[u], src) : 0;
                const uint32_t hs = (U & 1) ? __shfl_sync(0xffffffffu, ms, src) : 0u;
                const uint32_t hq = (U & 2) ? __shfl_sync(0xffffffffu, mp, src) : 0u;
                const uint32_t ho = (U & 4) ? __shfl_sync(0xffffffffu, mo, src) : 0u;
                int k = -1;
                if (m != 0) {
                    uint32_t h = s_msk[m];
                    if (m & 1) h ^= hs;
                    if (m & 2) h ^= kb_rotl(hq, 11);
                    if (m & 4) h ^= kb_rotl(ho, 22);
                    const uint32_t d = s_disp[kb_bucket(h, a.nb)];
                    const Entry en = s_tab[kb_slot(a.hp, h, d, a.ns)];
                    const bool hit = (en.mask_kid >> 28) == m && (!(m & 1) || en.s == ts) &&
                                     (!(m & 2) || en.p == tp) && (!(m & 4) || en.o == to);
                    k = hit ? (en.mask_kid & 0x0FFFFFFF) : -1;
                }
                if (!__any_sync(0xffffffffu, k >= 0)) continue;
                const unsigned peers = __match_any_sync(0xffffffffu, k);
                if (k >= 0) {
                    const uint32_t cc = cnt[k];
                    if (WRITE) {
                        const uint32_t r = cc + __popc(peers & lt);
                        a.arena[a.abs32 ? (int64_t)r : a.off[k] + r] = (int32_t)(b0 + u * 32 + src);
                    }
                    __syncwarp(peers);
                    if (lane == (unsigned)(__ffs(peers) - 1)) cnt[k] = cc + __popc(peers);
                }
                __syncwarp();
            }
            __syncwarp();  // the next slot rewrites the queue
        }
    }
    __syncwarp();
    if (!WRITE)
        for (int k = lane; k < a.kids; k += 32) row[k] = cnt[k];
}

// counts[w][k] -> exclusive prefix over w for each k; rows[k] = total of k.
// Block: 32 key ids (lanes) x 8 ranges of warps (the block's warps).
__global__ void __launch_bounds__(256) k_batch_scan(uint32_t *counts, int64_t GW, int kids, int64_t *rows) {
    __shared__ uint32_t s_sum[8][32];
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    const int64_t per = (GW + 7) / 8;
    const int64_t b = min((int64_t)w * per, GW), e = min(b + per, GW);
    uint32_t sum = 0;
    if (k < kids)
        for (int64_t g = b; g < e; ++g) sum += counts[g * kids + k];
    s_sum[w][lane] = sum;
    __syncthreads();
    uint32_t run = 0;
    for (unsigned v = 0; v < w; ++v) run += s_sum[v][lane];
    if (k < kids) {
        for (int64_t g = b; g < e; ++g) {
            const uint32_t c = counts[g * kids + k];
            counts[g * kids + k] = run;
            run += c;
        }
        if (w == 7) rows[k] = run;
    }
}

// Kernel shapes the autotuner chooses among.
enum Shape {
    SH_DIRECT = TID_BATCH_DIRECT,
    SH_DIRECT_SKIP = TID_BATCH_DIRECT_SKIP,
    SH_QUEUE4 = TID_BATCH_QUEUE4,
    SH_QUEUE8 = TID_BATCH_QUEUE8,
    SH_COUNT = 4
};

template <int U, bool WRITE, int SH>
void *kernel_of() {
    if (SH == SH_DIRECT) return (void *)k_batch<U, WRITE, false>;
    if (SH == SH_DIRECT_SKIP) return (void *)k_batch<U, WRITE, true>;
    if (SH == SH_QUEUE4) return (void *)k_batch_q<U, WRITE, 4>;
    return (void *)k_batch_q<U, WRITE, 8>;
}

// resident CTAs of both passes of a shape with `smem` bytes of dynamic shared memory
template <int U, int SH>
int kb_grid(size_t smem, unsigned *grid) {
    static bool opted = false;
    void *kw = kernel_of<U, true, SH>(), *kc = kernel_of<U, false, SH>();
    if (!opted) {  // dynamic shared memory up to the opt-in limit less the kernel's static share
        int optin = 0, dev = 0;
        cudaGetDevice(&dev);
        TID_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem limit");
        for (void *k : {kw, kc}) {
            cudaFuncAttributes fa{};
            TID_TRY_CUDA(cudaFuncGetAttributes(&fa, k), "k_batch attributes");
            TID_TRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              optin - (int)fa.sharedSizeBytes),
                         "k_batch smem");
        }
        opted = true;
    }
    int v = 0, w = 0;
    TID_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kw, KB_THREADS, smem), "occupancy");
    TID_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&w, kc, KB_THREADS, smem), "occupancy");
    if (std::min(v, w) < 1) return fail(TID_ERR_CAPACITY, "tid_match_batch: %zu bytes of shared memory per CTA", smem);
    *grid = (unsigned)(std::min(v, w) * sm_count());
    return TID_OK;
}

template <int U, int SH>
int run_pass(cudaStream_t st, bool write, unsigned grid, size_t smem, const BatchArgs &a) {
    void *k = write ? kernel_of<U, true, SH>() : kernel_of<U, false, SH>();
    BatchArgs args = a;
    void *params[] = {(void *)&args};
    TID_TRY_CUDA(cudaLaunchKernel(k, dim3(grid), dim3(KB_THREADS), params, smem, st), "k_batch");
    return TID_OK;
}

#define KB_DISPATCH_U(SH, U, fn, ...)                                       \
    switch (U) {                                                          \
        case 1: return fn<1, SH>(__VA_ARGS__);                            \
        case 2: return fn<2, SH>(__VA_ARGS__);                            \
        case 3: return fn<3, SH>(__VA_ARGS__);                            \
        case 4: return fn<4, SH>(__VA_ARGS__);                            \
        case 5: return fn<5, SH>(__VA_ARGS__);                            \
        case 6: return fn<6, SH>(__VA_ARGS__);                            \
        default: return fn<7, SH>(__VA_ARGS__);                           \
    }
#define KB_DISPATCH(shape, U, fn, ...)                                              \
    switch (shape) {                                                               \
        case SH_DIRECT: KB_DISPATCH_U(SH_DIRECT, U, fn, __VA_ARGS__)               \
        case SH_DIRECT_SKIP: KB_DISPATCH_U(SH_DIRECT_SKIP, U, fn, __VA_ARGS__)     \
        case SH_QUEUE4: KB_DISPATCH_U(SH_QUEUE4, U, fn, __VA_ARGS__)               \
        default: KB_DISPATCH_U(SH_QUEUE8, U, fn, __VA_ARGS__)                      \
    }

int grid_of(int U, int shape, size_t smem, unsigned *grid) { KB_DISPATCH(shape, U, kb_grid, smem, grid) }

int pass_of(int U, int shape, cudaStream_t st, bool write, unsigned grid, size_t smem, const BatchArgs &a) {
    KB_DISPATCH(shape, U, run_pass, st, write, grid, smem, a)
}

int slots_of(int shape) { return shape == SH_QUEUE4 ? 4 : 8; }  // 32-triple slots per iteration

using Key = std::tuple<int, int32_t, int32_t, int32_t>;  // mask, s, p, o (0 where unbound)

// Hash-and-displace table of `keys` (key id = position): buckets in decreasing
// size each take the first displacement that puts all their keys on free
// slots.  Returns false if some bucket finds none (the caller changes seed).
bool build_table(const std::vector<Key> &keys, const HashParams &hp, uint32_t nb, uint32_t ns, std::vector<Entry> &tab,
                 std::vector<uint16_t> &disp) {
    const int K = (int)keys.size();
    std::vector<uint32_t> h(K);
    std::vector<std::vector<int>> bucket(nb);
    for (int k = 0; k < K; ++k) {
        int m;
        int32_t s, p, o;
        std::tie(m, s, p, o) = keys[k];
        h[k] = kb_hash(hp, m, (uint32_t)s, (uint32_t)p, (uint32_t)o);
        bucket[kb_bucket(h[k], nb)].push_back(k);
    }
    std::vector<uint32_t> order(nb);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return bucket[x].size() > bucket[y].size(); });
    tab.assign(ns, Entry{0, 0, 0, -1});
    disp.assign(nb, 0);
    std::vector<char> used(ns, 0);
    std::vector<uint32_t> pos;
    for (uint32_t b : order) {
        const auto &ks = bucket[b];
        if (ks.empty()) break;
        bool placed = false;
        for (uint32_t d = 0; d < 65536 && !placed; ++d) {
            pos.clear();
            bool ok = true;
            for (int k : ks) {
                const uint32_t sl = kb_slot(hp, h[k], d, ns);
                if (used[sl] || std::find(pos.begin(), pos.end(), sl) != pos.end()) {
                    ok = false;
                    break;
                }
                pos.push_back(sl);
            }
            if (!ok) continue;
            for (size_t j = 0; j < ks.size(); ++j) {
                int m;
                int32_t s, p, o;
                std::tie(m, s, p, o) = keys[ks[j]];
                used[pos[j]] = 1;
                tab[pos[j]] = Entry{s, p, o, (m << 28) | ks[j]};
            }
            disp[b] = (uint16_t)d;
            placed = true;
        }
        if (!placed) return false;
    }
    return true;
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

// One sub-batch: key ids 0..K-1; sets[k] receives key id k's list.
// The host-side plan of one sub-batch: its keys (key id = position), the
// perfect-hash table with its parameters, and the prefilter.
struct SubPlan {
    std::vector<Key> keys;
    int U = 0;  // union of the keys' masks (the columns a pass reads)
    HashParams hp{};
    uint32_t nb = 0, ns = 0;
    std::vector<Entry> tab;
    std::vector<uint16_t> disp;
    std::vector<uint32_t> filt;
};

constexpr uint32_t KB_SEED = 0x243F6A88u;
constexpr int KB_SEEDS = 16;  // seeds tried before a sub-batch is split in two

// Table and prefilter for `keys`, trying seeds seed, seed + 1, ...; false if
// none of KB_SEEDS seeds gives a table (the caller splits the keys).
bool plan_keys(const std::vector<Key> &keys, uint32_t seed, SubPlan &sp, int *attempts) {
    const int kids = (int)keys.size();
    sp.keys = keys;
    sp.U = 0;
    for (auto &k : keys) sp.U |= std::get<0>(k);
    sp.nb = (uint32_t)std::max(1, (kids + 1) / 2);
    sp.ns = (uint32_t)(kids + kids / 8 + 8);
    bool built = false;
    for (int attempt = 0; attempt < KB_SEEDS && !built; ++attempt) {
        ++*attempts;
        sp.hp = hash_params(seed + (uint32_t)attempt);
        built = build_table(keys, sp.hp, sp.nb, sp.ns, sp.tab, sp.disp);
    }
    if (!built) return false;
    sp.filt.assign(3 * KB_FILTER_WORDS, 0u);
    for (auto &k : keys) {
        int m;
        int32_t kv[3];
        std::tie(m, kv[0], kv[1], kv[2]) = k;
        for (int c = 0; c < 3; ++c)
            if (m & (1 << c)) {
                const uint32_t f = kb_fentry(sp.hp, c, (uint32_t)kv[c]);
                sp.filt[c * KB_FILTER_WORDS + (f >> 3)] |= (1u << kb_fbit(c, m)) << ((f & 7u) * 4u);
            }
    }
    return true;
}

// Plans for keys[b, e): one sub-batch if a table is found, else the two halves.
// A table of one key always exists (any slot is free), so every batch of
// distinct keys is planned; false only if that ever failed.
bool plan_range(const std::vector<Key> &keys, size_t b, size_t e, uint32_t seed, std::vector<SubPlan> &plans,
                std::vector<size_t> &first, int *attempts) {
    SubPlan sp;
    const std::vector<Key> sub(keys.begin() + b, keys.begin() + e);
    if (plan_keys(sub, seed, sp, attempts)) {
        plans.push_back(std::move(sp));
        first.push_back(b);
        return true;
    }
    if (e - b < 2) return false;
    const size_t mid = b + (e - b) / 2;
    return plan_range(keys, b, mid, seed, plans, first, attempts) &&
           plan_range(keys, mid, e, seed, plans, first, attempts);
}

// Sub-batches of at most max_keys distinct keys; first[i] = key id of plans[i]'s key 0.
int plan_batch(const std::vector<Key> &keys, int max_keys, uint32_t seed, std::vector<SubPlan> &plans,
               std::vector<size_t> &first, int *attempts) {
    for (size_t b = 0; b < keys.size(); b += (size_t)max_keys)
        if (!plan_range(keys, b, std::min(keys.size(), b + (size_t)max_keys), seed, plans, first, attempts))
            return fail(TID_ERR_CAPACITY, "tid_match_batch: no key table for a single key");
    return TID_OK;
}

// Distinct (mask, key) pairs of a batch in first-seen order; kid_of[i] = key id
// of pattern i, or -1 for (?,?,?) or an empty store (answered by tid_match).
void batch_keys(const tid_pattern *pats, int q, bool empty_store, std::vector<Key> &keys, std::vector<int> &kid_of) {
    std::map<Key, int> id_of;
    kid_of.assign(q, -1);
    for (int i = 0; i < q; ++i) {
        const int m = (pats[i].s != 0) | ((pats[i].p != 0) << 1) | ((pats[i].o != 0) << 2);
        if (m == 0 || empty_store) continue;
        const Key key = std::make_tuple(m, pats[i].s, pats[i].p, pats[i].o);
        auto it = id_of.find(key);
        if (it == id_of.end()) {
            it = id_of.emplace(key, (int)keys.size()).first;
            keys.push_back(key);
        }
        kid_of[i] = it->second;
    }
}

// Device buffers of one sub-batch's table, prefilter and count matrix.
struct Uploaded {
    Entry *tab = nullptr;
    uint16_t *disp = nullptr;
    uint32_t *filt = nullptr;
    uint32_t *counts = nullptr;
    int64_t *off = nullptr;
};

int upload_plan(tid_ctx *ctx, Scratch &s, const SubPlan &sp, int64_t GW, Uploaded *u) {
    const int kids = (int)sp.keys.size();
    TID_TRY(s.get(&u->tab, sp.ns));
    TID_TRY(s.get(&u->disp, sp.nb));
    TID_TRY(s.get(&u->filt, 3 * KB_FILTER_WORDS));
    TID_TRY(s.get(&u->counts, (size_t)kids * GW));
    TID_TRY(s.get(&u->off, kids));
    cudaStream_t st = ctx->stream;
    TID_TRY_CUDA(cudaMemcpyAsync(u->tab, sp.tab.data(), sizeof(Entry) * sp.ns, cudaMemcpyHostToDevice, st),
                 "batch table");
    TID_TRY_CUDA(cudaMemcpyAsync(u->disp, sp.disp.data(), sizeof(uint16_t) * sp.nb, cudaMemcpyHostToDevice, st),
                 "batch table");
    TID_TRY_CUDA(cudaMemcpyAsync(u->filt, sp.filt.data(), sizeof(uint32_t) * 3 * KB_FILTER_WORDS,
                                 cudaMemcpyHostToDevice, st),
                 "batch prefilter");
    return TID_OK;
}

BatchArgs batch_args(const tid_store *st, const SubPlan &sp, const Uploaded &u, int64_t slice) {
    BatchArgs a{};
    a.S = st->s;
    a.P = st->p;
    a.O = st->o;
    a.n = st->n;
    a.slice = slice;
    a.kids = (int)sp.keys.size();
    a.hp = sp.hp;
    a.nb = sp.nb;
    a.ns = sp.ns;
    a.table = u.tab;
    a.disp = u.disp;
    a.filter = u.filt;
    a.counts = u.counts;
    return a;
}

// triples per warp slice: the store split evenly over GW warps, in whole iterations
int64_t slice_of(int64_t n, int64_t GW, int shape) {
    const int64_t gran = 32 * slots_of(shape);
    return std::max<int64_t>(gran, ceil_div(ceil_div(n, GW), gran) * gran);
}

// ---- autotuner ------------------------------------------------------------------
//
// Chooses, per (GPU, store size, masks read, log2 of the distinct keys), the
// kernel shape (direct lookups of every present mask, with or without warp
// skips of masks no lane may answer; or the candidate queue with 4 or 8 slots
// in flight) and the sub-batch size (1920 keys: two CTAs per SM; 1152: three).
// Each candidate's count pass is timed on a prefix of the store (2^25 triples;
// CUDA events, best of two) with a table of the batch's first keys, and the
// candidate with the least (sub-batches x pass time) is kept for the process.
struct TuneKey {
    int device, U, kbits, nbits;
    bool operator<(const TuneKey &o) const {
        return std::tie(device, U, kbits, nbits) < std::tie(o.device, o.U, o.kbits, o.nbits);
    }
};
struct Choice {
    int shape = SH_QUEUE8;
    int max_keys = KB_MAX_KIDS;
};
std::mutex g_tune_mu;
std::map<TuneKey, Choice> g_tuned;

constexpr int64_t KB_TUNE_TRIPLES = 1 << 25;
constexpr int KB_SIZES[2] = {KB_MAX_KIDS, 1152};

int ilog2_ceil(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

int tune_batch(tid_ctx *ctx, const tid_store *st, const std::vector<Key> &keys, Choice *out, bool *tuned_now) {
    *tuned_now = false;
    int U = 0;
    for (auto &k : keys) U |= std::get<0>(k);
    const TuneKey key{ctx->device, U, ilog2_ceil((int64_t)keys.size()), ilog2_ceil(st->n)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *out = it->second;
            return TID_OK;
        }
    }
    Choice best;
    if (st->n >= KB_TUNE_TRIPLES / 4) {
        cudaStream_t stream = ctx->stream;
        cudaEvent_t ev[2];
        for (auto &e : ev) TID_TRY_CUDA(cudaEventCreate(&e), "tuner events");
        struct EvFree {
            cudaEvent_t *e;
            ~EvFree() {
                cudaEventDestroy(e[0]);
                cudaEventDestroy(e[1]);
            }
        } evf{ev};
        tid_store pre = *st;
        pre.n = std::min<int64_t>(st->n, KB_TUNE_TRIPLES);
        float best_cost = 1e30f;
        for (int si = 0; si < 2; ++si) {
            const int size = KB_SIZES[si];
            if (si > 0 && (int64_t)keys.size() <= KB_SIZES[0] && (int64_t)keys.size() <= size) break;
            const std::vector<Key> first(keys.begin(), keys.begin() + std::min<size_t>(keys.size(), size));
            SubPlan sp;
            int tries = 0;
            if (!plan_keys(first, KB_SEED, sp, &tries)) continue;
            const size_t smem = kb_smem_bytes((int)first.size(), sp.ns, sp.nb);
            const float subs = (float)ceil_div((int64_t)keys.size(), size);
            for (int shape = 0; shape < SH_COUNT; ++shape) {
                unsigned grid = 0;
                if (grid_of(U, shape, smem, &grid) != TID_OK) {
                    clear_error();
                    continue;
                }
                const int64_t GW = (int64_t)grid * KB_WARPS;
                Scratch sc(ctx);
                Uploaded up;
                TID_TRY(upload_plan(ctx, sc, sp, GW, &up));
                BatchArgs a = batch_args(&pre, sp, up, slice_of(pre.n, GW, shape));
                float t = 1e30f;
                for (int rep = 0; rep < 2; ++rep) {
                    TID_TRY_CUDA(cudaEventRecord(ev[0], stream), "tuner timing");
                    TID_TRY(pass_of(U, shape, stream, false, grid, smem, a));
                    TID_TRY_CUDA(cudaEventRecord(ev[1], stream), "tuner timing");
                    TID_TRY_CUDA(cudaEventSynchronize(ev[1]), "tuner timing");
                    float ms = 0.f;
                    TID_TRY_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]), "tuner timing");
                    t = std::min(t, ms);
                }
                if (subs * t < best_cost) {
                    best_cost = subs * t;
                    best.shape = shape;
                    best.max_keys = size;
                }
            }
        }
        *tuned_now = true;
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best;
    *out = best;
    return TID_OK;
}

// The sub-batches on the device: every count pass and scan first, one
// synchronisation for all the list sizes, then every write pass.  Key id
// first[b] + k receives by_kid[first[b] + k].
int run_batch(tid_ctx *ctx, const tid_store *st, const std::vector<SubPlan> &plans, const std::vector<size_t> &first,
              int shape, std::vector<tid_set *> &by_kid) {
    cudaStream_t stream = ctx->stream;
    const size_t nsub = plans.size();
    struct Sub {
        size_t smem = 0;
        unsigned grid = 0;
        int64_t GW = 0;
        Uploaded up;
        BatchArgs a{};
        SharedBlock *sb = nullptr;
        std::vector<int64_t> tot, off;
    };
    std::vector<Sub> subs(nsub);
    Scratch s(ctx);
    auto give_up = [&](int code) {
        for (auto &b : subs)
            if (b.sb) {
                if (b.sb->ptr[0]) dev_free(ctx, b.sb->ptr[0]);
                if (b.sb->ptr[1]) dev_free(ctx, b.sb->ptr[1]);
                delete b.sb;
                b.sb = nullptr;
            }
        return code;
    };
    int rc = TID_OK;
    for (size_t b = 0; b < nsub; ++b) {
        const SubPlan &sp = plans[b];
        Sub &x = subs[b];
        const int kids = (int)sp.keys.size();
        x.smem = kb_smem_bytes(kids, sp.ns, sp.nb);
        if ((rc = grid_of(sp.U, shape, x.smem, &x.grid)) != TID_OK) return give_up(rc);
        x.GW = (int64_t)x.grid * KB_WARPS;
        x.sb = new (std::nothrow) SharedBlock();
        if (!x.sb) return give_up(fail(TID_ERR_OOM, "host allocation"));
        // the row counts live as long as the lists: both are the sets' shared block
        if ((rc = dev_alloc(ctx, &x.sb->ptr[0], sizeof(int64_t) * kids)) != TID_OK) return give_up(rc);
        if ((rc = upload_plan(ctx, s, sp, x.GW, &x.up)) != TID_OK) return give_up(rc);
        x.a = batch_args(st, sp, x.up, slice_of(st->n, x.GW, shape));
        if ((rc = pass_of(sp.U, shape, stream, false, x.grid, x.smem, x.a)) != TID_OK) return give_up(rc);
        k_batch_scan<<<(unsigned)ceil_div(kids, 32), 256, 0, stream>>>(x.up.counts, x.GW, kids,
                                                                       (int64_t *)x.sb->ptr[0]);
        if ((rc = launch_check("k_batch_scan")) != TID_OK) return give_up(rc);
        x.tot.resize(kids);
        cudaError_t ce = cudaMemcpyAsync(x.tot.data(), x.sb->ptr[0], sizeof(int64_t) * kids, cudaMemcpyDeviceToHost,
                                         stream);
        if (ce != cudaSuccess) return give_up(fail_cuda(ce, "batch totals"));
    }
    cudaError_t ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess) return give_up(fail_cuda(ce, "batch totals"));
    if ((rc = check_ctx_error(ctx)) != TID_OK) return give_up(rc);
    for (size_t b = 0; b < nsub; ++b) {
        Sub &x = subs[b];
        const int kids = (int)plans[b].keys.size();
        x.off.resize(kids);
        int64_t total = 0;
        for (int k = 0; k < kids; ++k) {  // lists start on 64-byte boundaries
            x.off[k] = total;
            total += (x.tot[k] + 15) / 16 * 16;
        }
        if ((rc = dev_alloc(ctx, &x.sb->ptr[1], sizeof(int32_t) * std::max<int64_t>(total, 16))) != TID_OK)
            return give_up(rc);
        ce = cudaMemcpyAsync(x.up.off, x.off.data(), sizeof(int64_t) * kids, cudaMemcpyHostToDevice, stream);
        if (ce != cudaSuccess) return give_up(fail_cuda(ce, "batch offsets"));
        x.a.arena = (int32_t *)x.sb->ptr[1];
        x.a.off = x.up.off;
        x.a.abs32 = total < ((int64_t)1 << 32) ? 1 : 0;
        if ((rc = pass_of(plans[b].U, shape, stream, true, x.grid, x.smem, x.a)) != TID_OK) return give_up(rc);
    }
    // hand each sub-batch's block to its sets (the last set freed releases it)
    for (size_t b = 0; b < nsub; ++b) {
        Sub &x = subs[b];
        const int kids = (int)plans[b].keys.size();
        int32_t *arena = (int32_t *)x.sb->ptr[1];
        int64_t *d_rows = (int64_t *)x.sb->ptr[0];
        for (int k = 0; k < kids; ++k) {
            rc = set_view(ctx, x.sb, arena + x.off[k], d_rows + k, x.tot[k], &by_kid[first[b] + k]);
            if (rc != TID_OK) break;
        }
        if (rc != TID_OK) {
            int made = 0;
            for (int k = 0; k < kids; ++k) made += by_kid[first[b] + k] != nullptr;
            if (made == 0) {  // nothing holds this block yet
                dev_free(ctx, x.sb->ptr[0]);
                dev_free(ctx, x.sb->ptr[1]);
                delete x.sb;
            }
            x.sb = nullptr;
            for (size_t c = b + 1; c < nsub; ++c) {  // blocks no set holds
                dev_free(ctx, subs[c].sb->ptr[0]);
                dev_free(ctx, subs[c].sb->ptr[1]);
                delete subs[c].sb;
                subs[c].sb = nullptr;
            }
            for (auto &h : by_kid) {  // the caller frees nothing: release every set made here
                if (h) set_free(h);
                h = nullptr;
            }
            return rc;
        }
        x.sb = nullptr;
    }
    return TID_OK;
}

}  // namespace
}  // namespace tid

using namespace tid;

extern "C" int tid_match_batch(tid_ctx *ctx, const tid_store *st, const tid_pattern *pats, int q, tid_set **outs) {
    clear_error();
    tid::Range nvtx_range("tid_match_batch");
    if (!ctx || !st || (q > 0 && (!pats || !outs))) return fail(TID_ERR_ARG, "tid_match_batch: null argument");
    if (q < 0) return fail(TID_ERR_ARG, "tid_match_batch: q = %d", q);
    if (st->ctx != ctx) return fail(TID_ERR_ARG, "tid_match_batch: store belongs to another context");
    for (int i = 0; i < q; ++i) outs[i] = nullptr;
    for (int i = 0; i < q; ++i)
        if (pats[i].s < 0 || pats[i].p < 0 || pats[i].o < 0)
            return fail(TID_ERR_ID, "tid_match_batch: negative ID in pattern %d", i);
    DeviceGuard g(ctx->device);
    // distinct (mask, key) -> key id; (?,?,?) and an empty store go through tid_match
    std::vector<Key> keys;
    std::vector<int> kid_of;
    batch_keys(pats, q, st->n == 0, keys, kid_of);
    std::vector<SubPlan> plans;
    std::vector<size_t> first;
    int attempts = 0;
    Choice ch;
    bool tuned_now = false;
    int rc = keys.empty() ? TID_OK : tune_batch(ctx, st, keys, &ch, &tuned_now);
    if (rc == TID_OK) rc = plan_batch(keys, ch.max_keys, KB_SEED, plans, first, &attempts);
    std::vector<tid_set *> by_kid(keys.size(), nullptr);
    if (rc == TID_OK && !plans.empty()) {
        ctx->batch_shape = ch.shape;
        ctx->batch_keys = ch.max_keys;
        ctx->batch_subs = (int)plans.size();
        rc = run_batch(ctx, st, plans, first, ch.shape, by_kid);
    }
    // the first pattern of a key id takes its set, equal patterns get views of the same list
    std::vector<bool> taken(keys.size(), false);
    for (int i = 0; i < q && rc == TID_OK; ++i) {
        const int k = kid_of[i];
        if (k < 0) {
            rc = tid_match(ctx, st, pats[i], &outs[i]);
        } else if (!taken[k]) {
            outs[i] = by_kid[k];
            taken[k] = true;
        } else {
            const tid_set *src = by_kid[k];
            rc = set_view(ctx, src->shared, src->col[0], src->d_rows, src->rows_known, &outs[i]);
        }
    }
    if (rc != TID_OK) {
        for (int i = 0; i < q; ++i) {
            if (outs[i] && (kid_of[i] < 0 || outs[i] != by_kid[kid_of[i]])) set_free(outs[i]);
            outs[i] = nullptr;
        }
        for (size_t k = 0; k < by_kid.size(); ++k) set_free(by_kid[k]);
        return rc;
    }
    return TID_OK;
}

// Host-only check of the batch's key tables (no device, no context): the same
// planning as tid_match_batch, then every key is looked up the way the kernel
// does -- its prefilter bits, bucket, displacement and slot -- and must find its
// own entry and key id; no two keys may share a slot.
extern "C" int tid_batch_table_check(const tid_pattern *pats, int q, uint32_t seed, int *attempts,
                                     int *sub_batches) {
    clear_error();
    if (q < 0 || (q > 0 && !pats)) return fail(TID_ERR_ARG, "tid_batch_table_check: bad patterns");
    for (int i = 0; i < q; ++i)
        if (pats[i].s < 0 || pats[i].p < 0 || pats[i].o < 0)
            return fail(TID_ERR_ID, "tid_batch_table_check: negative ID in pattern %d", i);
    std::vector<Key> keys;
    std::vector<int> kid_of;
    batch_keys(pats, q, false, keys, kid_of);
    std::vector<SubPlan> plans;
    std::vector<size_t> first;
    int tries = 0;
    TID_TRY(plan_batch(keys, KB_MAX_KIDS, seed, plans, first, &tries));
    size_t covered = 0;
    for (size_t b = 0; b < plans.size(); ++b) {
        const SubPlan &sp = plans[b];
        if (first[b] != covered) return fail(TID_ERR_CAPACITY, "sub-batch %zu does not follow its predecessor", b);
        covered += sp.keys.size();
        std::vector<int> owner(sp.ns, -1);
        for (int k = 0; k < (int)sp.keys.size(); ++k) {
            int m;
            int32_t kv[3];
            std::tie(m, kv[0], kv[1], kv[2]) = sp.keys[k];
            uint32_t e3[3];
            for (int c = 0; c < 3; ++c) {
                const uint32_t f = kb_fentry(sp.hp, c, (uint32_t)kv[c]);
                e3[c] = (sp.filt[c * KB_FILTER_WORDS + (f >> 3)] >> ((f & 7u) * 4u)) & 0xFu;
            }
            // a triple with this key's values at the bound slots, whatever it holds elsewhere
            for (uint32_t other = 0; other < 16; ++other) {
                const uint32_t cand = kb_candidates((m & 1) ? e3[0] : other, (m & 2) ? e3[1] : other,
                                                    (m & 4) ? e3[2] : other);
                if (!((cand >> m) & 1)) return fail(TID_ERR_CAPACITY, "prefilter drops key %d of sub-batch %zu", k, b);
            }
            const uint32_t h = kb_hash(sp.hp, m, (uint32_t)kv[0], (uint32_t)kv[1], (uint32_t)kv[2]);
            const uint32_t sl = kb_slot(sp.hp, h, sp.disp[kb_bucket(h, sp.nb)], sp.ns);
            const Entry &en = sp.tab[sl];
            if (en.mask_kid != ((m << 28) | k) || ((m & 1) && en.s != kv[0]) || ((m & 2) && en.p != kv[1]) ||
                ((m & 4) && en.o != kv[2]))
                return fail(TID_ERR_CAPACITY, "key %d of sub-batch %zu not found at its slot", k, b);
            if (owner[sl] >= 0) return fail(TID_ERR_CAPACITY, "keys %d and %d share a slot", owner[sl], k);
            owner[sl] = k;
        }
    }
    if (covered != keys.size()) return fail(TID_ERR_CAPACITY, "sub-batches hold %zu of %zu keys", covered, keys.size());
    if (attempts) *attempts = tries;
    if (sub_batches) *sub_batches = (int)plans.size();
    return TID_OK;
}

extern "C" int tid_batch_tuning(const tid_ctx *ctx, int32_t *shape, int32_t *keys_per_sub_batch,
                                int32_t *sub_batches) {
    clear_error();
    if (!ctx) return fail(TID_ERR_ARG, "tid_batch_tuning: null context");
    if (shape) *shape = ctx->batch_shape;
    if (keys_per_sub_batch) *keys_per_sub_batch = ctx->batch_keys;
    if (sub_batches) *sub_batches = ctx->batch_subs;
    return TID_OK;
}
