// K4: stable LSD radix sort of tuple rows, and the canonical form of a set.
//
// The paper sorts every result vector before joining and merges the final
// results to keep distinct values (Section 4.3); it used a library mergesort.
// When the columns' value ranges fit 64 bits together (the usual case: entity
// IDs need ~23 bits), each row is packed into one 32- or 64-bit key -- column
// 0 most significant, each field rebased to (x - min) and as wide as
// (max - min) needs -- and the keys alone are radix sorted, then unpacked (and
// adjacent duplicates dropped) in one streaming pass.  Otherwise a row
// permutation is sorted: for each key column from the last to the first, the
// (key, row) pairs are radix sorted stably, so the final permutation orders
// rows lexicographically; again only the bits that vary are sorted.
//
// One digit pass = per-tile histograms (k_tile_hist) + a scan of each digit's
// tile counts (k_digit_scan, one CTA per digit) + one ranking-and-scatter
// launch (k_onesweep): tiles of 4096
// keys rank stably (the lanes of a warp with equal digits found by a match
// instruction or by eight ballots, alternately, the first lane of each group
// adding its size to a shared counter)
// and scatter through shared memory so runs of equal digits are written
// contiguously, at the scanned offsets.  No tile
// waits for another: a one-launch form whose tiles took each bin's offset by a
// decoupled look-back over earlier tiles (Adinets and Merrill, "Onesweep",
// 2022) waited there longer than its tiles worked, every tile walking back
// through all the tiles in flight.  Bytes per digit: w n read twice (the
// histogram read mostly from L2) + w n written, w = key bytes (4 or 8; 4 + 4
// with the permutation), plus one read of the columns for packing.
//
// Sets of at most 4096 packed rows skip the passes: one CTA loads the keys into
// shared memory, bitonic-sorts them, flags and block-scans the distinct ones
// and unpacks them -- one launch, as the many small sets of a plan need.

#include <algorithm>

#include "tid_internal.cuh"
#include "ops.cuh"

namespace tid {

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
// Shape of a digit pass: keys per thread (a tile is 256 threads' keys) and the
// CTAs per SM the scatter pass is compiled for.  The scatter pass is
// latency-bound (shared-memory round trips per key), so resident CTAs matter:
//  - keys-only 32-bit sorts: 16 keys, four CTAs (64 registers; 26 % faster
//    than three CTAs on 32M rows);
//  - 64-bit keys, at most RS_SMALL keys: 12 keys, four CTAs (the 23.6M-row
//    projection 14 % faster, the 12M-row bind sort faster too);
//  - larger 64-bit sorts and the (key, row) pairs of the permutation sort:
//    16 keys, three CTAs (12 keys at four CTAs measured 4-8 % slower on 32M
//    to 60M keys).
// 32 keys per thread at two CTAs measured slower for every size.
constexpr int64_t RS_SMALL = 24ll << 20;
// Sorts of at most this many tiles skip the digit-scan launch: each scatter
// CTA sums its digit's row of tile counts (the many small sorts of a plan).
constexpr unsigned RS_FEW_TILES = 32;
constexpr int RS_BINS = 256;

struct ColPtrs {
    const int32_t *c[TID_MAX_COLS];
};
struct MutColPtrs {
    int32_t *c[TID_MAX_COLS];
};


__device__ __forceinline__ uint32_t order_key(int32_t x) { return (uint32_t)x ^ 0x80000000u; }

// The streaming kernels below (k_minmax, k_prep, k_pack, k_unpack, k_gather)
// take EW_U elements per thread per step, a block's EW_U * blockDim.x
// consecutive elements at a time, and issue all of a step's loads before using
// them: one 4-byte load per thread in flight did not cover HBM latency.
constexpr int EW_U = 4;
constexpr int EW_THREADS = 256;

__device__ __forceinline__ int64_t ew_first() { return (int64_t)blockIdx.x * (EW_THREADS * EW_U) + threadIdx.x; }
__device__ __forceinline__ int64_t ew_stride() { return (int64_t)gridDim.x * (EW_THREADS * EW_U); }

// per-column min and max in sort order (flipped sign bit)
__global__ void __launch_bounds__(EW_THREADS) k_minmax(ColPtrs cols, int k, int64_t n, uint32_t *__restrict__ mn,
                                                       uint32_t *__restrict__ mx) {
    uint32_t lo[TID_MAX_COLS], hi[TID_MAX_COLS];
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        lo[c] = 0xFFFFFFFFu;
        hi[c] = 0u;
    }
    for (int64_t i0 = ew_first(); i0 < n; i0 += ew_stride()) {
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c >= k) continue;
            uint32_t v[EW_U];
#pragma unroll
            for (int u = 0; u < EW_U; ++u) {
                const int64_t i = i0 + u * EW_THREADS;
                v[u] = i < n ? order_key(cols.c[c][i]) : order_key(cols.c[c][i0]);
            }
#pragma unroll
            for (int u = 0; u < EW_U; ++u) {
                lo[c] = min(lo[c], v[u]);
                hi[c] = max(hi[c], v[u]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < TID_MAX_COLS; ++c) {
        if (c >= k) continue;
        uint32_t a = lo[c], b = hi[c];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            a = min(a, __shfl_xor_sync(0xffffffffu, a, d));
            b = max(b, __shfl_xor_sync(0xffffffffu, b, d));
        }
        if ((threadIdx.x & 31) == 0) {  // skip an atomic that cannot tighten the bound
            if (a < __ldcg(mn + c)) atomicMin(mn + c, a);
            if (b > __ldcg(mx + c)) atomicMax(mx + c, b);
        }
    }
}


// keys[i] = order_key(col[src(i)]) - base, vals[i] = src(i), src = perm ? perm[i] : i
__global__ void __launch_bounds__(EW_THREADS) k_prep(const int32_t *__restrict__ col, const int32_t *__restrict__ perm,
                                                     int64_t n, uint32_t base, uint32_t *__restrict__ keys,
                                                     int32_t *__restrict__ vals) {
    for (int64_t i0 = ew_first(); i0 < n; i0 += ew_stride()) {
        int32_t s[EW_U], x[EW_U];
#pragma unroll
        for (int u = 0; u < EW_U; ++u) {
            const int64_t i = i0 + u * EW_THREADS;
            s[u] = i < n ? (perm ? perm[i] : (int32_t)i) : 0;
        }
#pragma unroll
        for (int u = 0; u < EW_U; ++u) x[u] = i0 + u * EW_THREADS < n ? col[s[u]] : 0;
#pragma unroll
        for (int u = 0; u < EW_U; ++u) {
            const int64_t i = i0 + u * EW_THREADS;
            if (i < n) {
                keys[i] = order_key(x[u]) - base;
                vals[i] = s[u];
            }
        }
    }
}

__global__ void k_iota32(int32_t *__restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)i;
}

// Per-tile histogram of one digit: hist[d * tiles + t] = keys of tile t (ITEMS x 256
// keys) whose digit at `shift` is d.  Per-warp counters in shared memory (a
// whole warp on one digit is one add).
template <typename K, int ITEMS>
__global__ void __launch_bounds__(RS_THREADS) k_tile_hist(const K *__restrict__ keys, int64_t n, int shift,
                                                          uint32_t *__restrict__ hist, unsigned tiles) {
    __shared__ uint32_t s_h[RS_WARPS][RS_BINS];
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * (RS_THREADS * ITEMS);
    K k[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = base + j * RS_THREADS + threadIdx.x;
        k[j] = i < n ? keys[i] : (K)0;
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = base + j * RS_THREADS + threadIdx.x;
        const bool valid = i < n;
        const unsigned d = valid ? (unsigned)(k[j] >> shift) & 0xFFu : 0x100u;
        const unsigned d0 = __shfl_sync(0xffffffffu, d, 0);
        if (__all_sync(0xffffffffu, d == d0)) {
            if (lane == 0 && d0 < 0x100u) s_h[warp][d0] += 32u;
        } else if (valid) {
            atomicAdd(&s_h[warp][d], 1u);
        }
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) c += s_h[w][threadIdx.x];
    hist[(size_t)threadIdx.x * tiles + blockIdx.x] = c;
}

// In place: row d of the per-tile histograms (hist[d * tiles + t]) becomes its
// exclusive scan over the tiles, and tot[d] the row's total.  One CTA per
// digit, stepping through its row 1024 tiles at a time with a carry.
__global__ void __launch_bounds__(1024) k_digit_scan(uint32_t *__restrict__ hist, unsigned tiles,
                                                     uint32_t *__restrict__ tot) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_chunk;
    uint32_t *row = hist + (size_t)blockIdx.x * tiles;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (unsigned b = 0; b < tiles; b += 1024) {
        const unsigned t = b + threadIdx.x;
        const uint32_t v = t < tiles ? row[t] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = s_w[lane];
            uint32_t y = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
                if ((int)lane >= o) y += z;
            }
            s_w[lane] = y - w;
            if (lane == 31) s_chunk = y;
        }
        __syncthreads();
        if (t < tiles) row[t] = carry + s_w[warp] + x - v;
        carry += s_chunk;
        __syncthreads();  // s_w and s_chunk are rewritten by the next chunk
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// The offset of (digit d, tile t) is the keys of smaller digits (the exclusive
// scan of tot) plus offs[d * tiles + t], the row-scanned per-tile histograms
// (k_tile_hist, k_digit_scan), so no tile waits for another.
template <typename K, bool HAS_VAL, int ITEMS, int MINB>
__global__ void __launch_bounds__(RS_THREADS, MINB)
k_onesweep(const K *__restrict__ kin, const int32_t *__restrict__ vin, K *__restrict__ kout, int32_t *__restrict__ vout,
           int64_t n, int shift, const uint32_t *__restrict__ offs, const uint32_t *__restrict__ tot, unsigned tiles) {
    __shared__ uint32_t s_wcnt[RS_WARPS][RS_BINS];
    __shared__ uint32_t s_gbase[RS_BINS];
    __shared__ uint32_t s_wsum[RS_WARPS], s_wtot[RS_WARPS];
    __shared__ K s_k[(RS_THREADS * ITEMS)];
    __shared__ int32_t s_v[HAS_VAL ? (RS_THREADS * ITEMS) : 1];

    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&s_wcnt[0][0])[i] = 0;
    const unsigned tile = blockIdx.x;
    {
        // this tile's first output position per digit (one digit per thread):
        // the keys of smaller digits (exclusive scan of tot) + this digit's
        // keys in earlier tiles
        const unsigned d = threadIdx.x;
        // tot == nullptr: the histograms were not scanned (a sort of at most
        // RS_FEW_TILES tiles); the digit's row is summed here instead
        uint32_t t = 0, pre = 0;
        if (tot) {
            t = tot[d];
            pre = offs[(size_t)d * tiles + tile];
        } else {
            for (unsigned u = 0; u < tiles; ++u) {
                const uint32_t c = offs[(size_t)d * tiles + u];
                t += c;
                pre += u < tile ? c : 0u;
            }
        }
        uint32_t x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) s_wtot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < RS_WARPS ? s_wtot[lane] : 0u;
            uint32_t y = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
                if ((int)lane >= o) y += z;
            }
            if (lane < RS_WARPS) s_wtot[lane] = y - w;
        }
        __syncthreads();
        s_gbase[d] = x - t + s_wtot[warp] + pre;
    }
    __syncthreads();
    const int64_t base = (int64_t)tile * (RS_THREADS * ITEMS);
    const int64_t wbase = base + (int64_t)warp * (ITEMS * 32);
    K k[ITEMS];
    uint32_t r[ITEMS / 2];  // ranks within the warp (< 32 ITEMS), two per register
    int32_t v[HAS_VAL ? ITEMS : 1];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        const bool valid = i < n;
        k[j] = valid ? kin[i] : (K)0;
        if (HAS_VAL) v[j] = valid ? vin[i] : 0;
    }
    // stable rank among this warp's rows with the same digit, in row order: the
    // first lane of each group of equal digits adds the group's size to the
    // warp's counter (the shared-memory atomic returns the count before it) and
    // the group reads that base from it -- no warp-wide wait between items,
    // so the items' counter updates overlap
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        const bool valid = i < n;
        // lanes with the same digit.  Two ways that load different pipes are
        // alternated over the items: the warp-wide match instruction (its
        // pipe alone held the kernel back when every item used it), and one
        // ballot per digit bit (ALU work: alone, the ALU pipe bounded it).
        unsigned peers;
        if ((j & 1) == 0) {
            peers = __match_any_sync(0xffffffffu, valid ? (unsigned)(k[j] >> shift) & 0xFFu : 0x100u);
        } else {
            const unsigned d = valid ? (unsigned)(k[j] >> shift) & 0xFFu : 0u;
            peers = __ballot_sync(0xffffffffu, valid);  // separates the tail's invalid lanes
            if (!valid) peers = ~peers;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const bool bit = (d >> b) & 1u;
                const unsigned bb = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bb : ~bb;
            }
        }
        const unsigned d = valid ? (unsigned)(k[j] >> shift) & 0xFFu : 0u;
        const int leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if (valid && lane == (unsigned)leader) b = atomicAdd(&s_wcnt[warp][d], (uint32_t)__popc(peers));
        b = __shfl_sync(0xffffffffu, b, leader);
        const uint32_t rank = b + __popc(peers & lt);
        if (j & 1) r[j >> 1] |= rank << 16;
        else r[j >> 1] = rank;
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
        // digit d's first position in the tile, folded into each warp's
        // counter (one shared load per key when scattering) and into the
        // digit's tile-to-output shift (one per key when writing out)
        const uint32_t tdig = x - run + s_wsum[warp];
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) s_wcnt[w][d] += tdig;
        s_gbase[d] -= tdig;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        if (i < n) {
            const unsigned d = (unsigned)(k[j] >> shift) & 0xFFu;
            const uint32_t lp = s_wcnt[warp][d] + ((r[j >> 1] >> (16 * (j & 1))) & 0xFFFFu);
            s_k[lp] = k[j];
            if (HAS_VAL) s_v[lp] = v[j];
        }
    }
    __syncthreads();
    const int cnt = (int)(n - base < (RS_THREADS * ITEMS) ? n - base : (RS_THREADS * ITEMS));
    for (int i = threadIdx.x; i < cnt; i += RS_THREADS) {
        const K kk = s_k[i];
        const unsigned d = (unsigned)(kk >> shift) & 0xFFu;
        const uint32_t gp = s_gbase[d] + (uint32_t)i;  // wraps modulo 2^32 to the right position
        kout[gp] = kk;
        if (HAS_VAL) vout[gp] = s_v[i];
    }
}

// packed key of a row: column 0 most significant; field c holds
// order_key(col_c) - min_c in bits [shift_c, shift_c + bits_c)
template <typename K>
__global__ void __launch_bounds__(EW_THREADS) k_pack(ColPtrs cols, int k, int64_t n, PackSpec ps,
                                                     K *__restrict__ keys) {
    for (int64_t i0 = ew_first(); i0 < n; i0 += ew_stride()) {
        K key[EW_U];
#pragma unroll
        for (int u = 0; u < EW_U; ++u) key[u] = 0;
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {  // a constant column (mask 0) has no field
            if (c >= k || !ps.mask[c]) continue;
            int32_t x[EW_U];
#pragma unroll
            for (int u = 0; u < EW_U; ++u) {
                const int64_t i = i0 + u * EW_THREADS;
                x[u] = i < n ? cols.c[c][i] : 0;
            }
#pragma unroll
            for (int u = 0; u < EW_U; ++u) key[u] |= (K)(order_key(x[u]) - ps.min[c]) << ps.shift[c];
        }
#pragma unroll
        for (int u = 0; u < EW_U; ++u) {
            const int64_t i = i0 + u * EW_THREADS;
            if (i < n) keys[i] = key[u];
        }
    }
}

// sorted packed keys -> k columns (no duplicate removal)
template <typename K>
__global__ void __launch_bounds__(EW_THREADS) k_unpack(const K *__restrict__ keys, int k, int64_t n, PackSpec ps,
                                                       MutColPtrs out) {
    for (int64_t i0 = ew_first(); i0 < n; i0 += ew_stride()) {
        K key[EW_U];
#pragma unroll
        for (int u = 0; u < EW_U; ++u) {
            const int64_t i = i0 + u * EW_THREADS;
            key[u] = i < n ? keys[i] : (K)0;
        }
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c >= k) continue;
#pragma unroll
            for (int u = 0; u < EW_U; ++u) {
                const int64_t i = i0 + u * EW_THREADS;
                const uint32_t f = ps.mask[c] ? (uint32_t)((key[u] >> ps.shift[c]) & ps.mask[c]) : 0u;
                if (i < n) out.c[c][i] = (int32_t)((f + ps.min[c]) ^ 0x80000000u);
            }
        }
    }
}

// Small sets (n <= SMALL_N rows) in one CTA: pack, bitonic sort in shared memory
// (padded to a power of two with the largest key), drop adjacent duplicates if
// asked (flags + block scan), unpack, and write the row count -- one launch
// instead of the passes of the device-wide sort.
constexpr int SMALL_N = 4096;
constexpr int SMALL_THREADS = 1024;

template <typename K>
__global__ void __launch_bounds__(SMALL_THREADS) k_small_canonical(ColPtrs cols, int k, int n, PackSpec ps,
                                                                   int dedupe, MutColPtrs out,
                                                                   int64_t *__restrict__ d_rows,
                                                                   int64_t *__restrict__ h_rows) {
    __shared__ K sk[SMALL_N];
    __shared__ uint32_t s_warp[SMALL_THREADS / 32];
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += SMALL_THREADS) {
        K key = ~(K)0;
        if (i < n) {
            key = 0;
#pragma unroll
            for (int c = 0; c < TID_MAX_COLS; ++c)
                if (c < k && ps.mask[c]) key |= (K)(order_key(cols.c[c][i]) - ps.min[c]) << ps.shift[c];
        }
        sk[i] = key;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P / 2; t += SMALL_THREADS) {
                const int i = 2 * t - (t & (stride - 1));  // lower index of the pair
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const K a = sk[i], b = sk[j];
                if ((a > b) == up) {
                    sk[i] = b;
                    sk[j] = a;
                }
            }
            __syncthreads();
        }
    }
    // each thread owns up to SMALL_N / SMALL_THREADS consecutive sorted rows
    constexpr int PER = SMALL_N / SMALL_THREADS;
    const int b = threadIdx.x * PER;
    bool keep[PER];
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = b + q;
        keep[q] = i < n && (!dedupe || i == 0 || sk[i] != sk[i - 1]);
        cnt += keep[q];
    }
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if ((int)lane >= d) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t base = 0;
    for (unsigned w = 0; w < warp; ++w) base += s_warp[w];
    uint32_t pos = base + x - cnt;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        if (!keep[q]) continue;
        const K key = sk[b + q];
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c >= k) continue;
            const uint32_t f = ps.mask[c] ? (uint32_t)((key >> ps.shift[c]) & ps.mask[c]) : 0u;
            out.c[c][pos] = (int32_t)((f + ps.min[c]) ^ 0x80000000u);
        }
        ++pos;
    }
    if (threadIdx.x == SMALL_THREADS - 1) {
        *d_rows = pos;
        *h_rows = pos;
    }
}

__global__ void __launch_bounds__(EW_THREADS) k_gather(ColPtrs in, int k, const int32_t *__restrict__ perm, int64_t n,
                                                       MutColPtrs out) {
    for (int64_t i0 = ew_first(); i0 < n; i0 += ew_stride()) {
        int64_t s[EW_U];
#pragma unroll
        for (int u = 0; u < EW_U; ++u) {
            const int64_t i = i0 + u * EW_THREADS;
            s[u] = i < n ? perm[i] : 0;
        }
#pragma unroll
        for (int c = 0; c < TID_MAX_COLS; ++c) {
            if (c >= k) continue;
            int32_t x[EW_U];
#pragma unroll
            for (int u = 0; u < EW_U; ++u) x[u] = i0 + u * EW_THREADS < n ? in.c[c][s[u]] : 0;
#pragma unroll
            for (int u = 0; u < EW_U; ++u) {
                const int64_t i = i0 + u * EW_THREADS;
                if (i < n) out.c[c][i] = x[u];
            }
        }
    }
}

__global__ void k_set_rows(int64_t *d_rows, int64_t *h_rows, int64_t n) {
    *d_rows = n;
    *h_rows = n;
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

// Per-column [min, max] in sort order (one kernel, one synchronisation).
static int column_ranges(tid_ctx *ctx, const int32_t *const *cols, int k, int64_t n, uint32_t *hmin, uint32_t *hmax) {
    cudaStream_t st = ctx->stream;
    Scratch s(ctx);
    uint32_t *mm = nullptr;
    TID_TRY(s.get(&mm, 2 * TID_MAX_COLS));
    ColPtrs cp{};
    for (int c = 0; c < k; ++c) cp.c[c] = cols[c];
    TID_TRY_CUDA(cudaMemsetAsync(mm, 0xFF, TID_MAX_COLS * 4, st), "memset");
    TID_TRY_CUDA(cudaMemsetAsync(mm + TID_MAX_COLS, 0, TID_MAX_COLS * 4, st), "memset");
    k_minmax<<<grid_for(n, EW_THREADS * EW_U, 8), EW_THREADS, 0, st>>>(cp, k, n, mm, mm + TID_MAX_COLS);
    TID_TRY(launch_check("k_minmax"));
    uint32_t both[2 * TID_MAX_COLS];
    TID_TRY_CUDA(cudaMemcpyAsync(both, mm, sizeof both, cudaMemcpyDeviceToHost, st), "copy min/max");
    TID_TRY_CUDA(cudaStreamSynchronize(st), "sync min/max");
    for (int c = 0; c < k; ++c) {
        hmin[c] = both[c];
        hmax[c] = both[TID_MAX_COLS + c];
    }
    return TID_OK;
}

static int range_bits(uint32_t lo, uint32_t hi) { return hi == lo ? 0 : 32 - __builtin_clz(hi - lo); }

// Each digit: per-tile histograms, one scan of the (digit, tile) counts, then
// the ranking and scatter at the scanned offsets.
template <typename K, bool HAS_VAL>
static int radix_passes(tid_ctx *ctx, K *&ka, K *&kb, int32_t *&pa, int32_t *&pb, int64_t n, int shift0,
                        int passes);

template <typename K, bool HAS_VAL, int ITEMS, int MINB>
static int radix_passes_shaped(tid_ctx *ctx, K *&ka, K *&kb, int32_t *&pa, int32_t *&pb, int64_t n, int shift0,
                               int passes) {
    const unsigned tiles = (unsigned)ceil_div(n, RS_THREADS * ITEMS);
    uint32_t *offs = nullptr;
    TID_TRY(dev_alloc(ctx, (void **)&offs, sizeof(uint32_t) * (size_t)RS_BINS * (tiles + 1)));
    uint32_t *tot = offs + (size_t)RS_BINS * tiles;
    int rc = TID_OK;
    for (int p = 0; p < passes && rc == TID_OK; ++p) {
        const int shift = shift0 + 8 * p;
        k_tile_hist<K, ITEMS><<<tiles, RS_THREADS, 0, ctx->stream>>>(ka, n, shift, offs, tiles);
        rc = launch_check("k_tile_hist");
        const bool scan = tiles > RS_FEW_TILES;  // else each scatter CTA sums its digits' rows itself
        if (rc == TID_OK && scan) {
            k_digit_scan<<<RS_BINS, 1024, 0, ctx->stream>>>(offs, tiles, tot);
            rc = launch_check("k_digit_scan");
        }
        if (rc == TID_OK) {
            k_onesweep<K, HAS_VAL, ITEMS, MINB><<<tiles, RS_THREADS, 0, ctx->stream>>>(ka, pa, kb, pb, n, shift, offs,
                                                                                scan ? tot : nullptr, tiles);
            rc = launch_check("k_onesweep");
        }
        std::swap(ka, kb);
        if (HAS_VAL) std::swap(pa, pb);
    }
    dev_free(ctx, offs);
    return rc;
}

template <typename K, bool HAS_VAL>
static int radix_passes(tid_ctx *ctx, K *&ka, K *&kb, int32_t *&pa, int32_t *&pb, int64_t n, int shift0,
                        int passes) {
    if constexpr (sizeof(K) == 4 && !HAS_VAL) {
        return radix_passes_shaped<K, HAS_VAL, 16, 4>(ctx, ka, kb, pa, pb, n, shift0, passes);
    } else if constexpr (sizeof(K) == 8) {
        if (n <= RS_SMALL) return radix_passes_shaped<K, HAS_VAL, 12, 4>(ctx, ka, kb, pa, pb, n, shift0, passes);
        return radix_passes_shaped<K, HAS_VAL, 16, 3>(ctx, ka, kb, pa, pb, n, shift0, passes);
    } else {
        return radix_passes_shaped<K, HAS_VAL, 16, 3>(ctx, ka, kb, pa, pb, n, shift0, passes);
    }
}

// Stable LSD sort of a row permutation by key columns, given their ranges.  The
// rows are already in order of the last `sorted_tail` key columns (taken in
// their order), so those passes are skipped: stable passes over the leading
// columns keep them in order within equal leading values.
static int sort_perm_ranges(tid_ctx *ctx, const int32_t *const *keys, int nk, int64_t n, const uint32_t *hmin,
                            const uint32_t *hmax, int32_t *perm, int sorted_tail = 0) {
    cudaStream_t st = ctx->stream;
    Scratch s(ctx);
    uint32_t *ka = nullptr, *kb = nullptr;
    int32_t *pa = nullptr, *pb = nullptr;
    bool have_perm = false;  // pa holds the current permutation
    for (int c = nk - 1 - sorted_tail; c >= 0; --c) {
        const int bits = range_bits(hmin[c], hmax[c]);
        if (bits == 0) continue;  // constant column: order unchanged
        const int passes = (bits + 7) / 8;
        if (!ka) {
            TID_TRY(s.get(&ka, n));
            TID_TRY(s.get(&kb, n));
            TID_TRY(s.get(&pa, n));
            TID_TRY(s.get(&pb, n));
        }
        k_prep<<<grid_for(n, EW_THREADS * EW_U, 8), EW_THREADS, 0, st>>>(keys[c], have_perm ? pa : nullptr, n, hmin[c], ka, pa);
        TID_TRY(launch_check("k_prep"));
        TID_TRY((radix_passes<uint32_t, true>(ctx, ka, kb, pa, pb, n, 0, passes)));
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

int sort_perm(tid_ctx *ctx, const int32_t *const *keys, int nk, int64_t n, int32_t *perm) {
    if (n <= 0) return TID_OK;
    if (nk < 0 || nk > TID_MAX_COLS) return fail(TID_ERR_ARG, "sort: %d key columns", nk);
    uint32_t hmin[TID_MAX_COLS] = {0}, hmax[TID_MAX_COLS] = {0};
    if (nk > 0) TID_TRY(column_ranges(ctx, keys, nk, n, hmin, hmax));
    return sort_perm_ranges(ctx, keys, nk, n, hmin, hmax, perm);
}

// Canonical form by sorting packed keys (all fields fit K): pack, keys-only
// digit passes over the occupied bits, then unpack (with distinct rows kept).
// The rows are already ordered by the low `sorted_bits` bits of their keys
// (the fields of trailing columns they are sorted by): the digit passes start
// above them.
template <typename K>
static int canonical_packed(tid_ctx *ctx, const int32_t *const *cols, int k, int64_t n, bool dedupe,
                            const PackSpec &ps, int total_bits, int sorted_bits, tid_set *set) {
    cudaStream_t st = ctx->stream;
    if (n <= SMALL_N) {
        ColPtrs cp{};
        MutColPtrs op{};
        for (int c = 0; c < k; ++c) {
            cp.c[c] = cols[c];
            op.c[c] = set->col[c];
        }
        k_small_canonical<K><<<1, SMALL_THREADS, 0, st>>>(cp, k, (int)n, ps, dedupe ? 1 : 0, op, set->d_rows,
                                                          set->slot.dev);
        TID_TRY(launch_check("k_small_canonical"));
        if (!dedupe) set->rows_known = n;
        return TID_OK;
    }
    Scratch s(ctx);
    K *ka = nullptr, *kb = nullptr;
    int32_t *none_a = nullptr, *none_b = nullptr;
    const int passes = (total_bits - sorted_bits + 7) / 8;
    TID_TRY(s.get(&ka, n));
    TID_TRY(s.get(&kb, n));
    ColPtrs cp{};
    for (int c = 0; c < k; ++c) cp.c[c] = cols[c];
    k_pack<K><<<grid_for(n, EW_THREADS * EW_U, 8), EW_THREADS, 0, st>>>(cp, k, n, ps, ka);
    TID_TRY(launch_check("k_pack"));
    TID_TRY((radix_passes<K, false>(ctx, ka, kb, none_a, none_b, n, sorted_bits, passes)));
    if (dedupe) return compact_unique_packed(ctx, ka, sizeof(K) == 8, k, n, ps, set);
    MutColPtrs op{};
    for (int c = 0; c < k; ++c) op.c[c] = set->col[c];
    k_unpack<K><<<grid_for(n, EW_THREADS * EW_U, 8), EW_THREADS, 0, st>>>(ka, k, n, ps, op);
    TID_TRY(launch_check("k_unpack"));
    return set_rows_const(set, n);
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
    k_gather<<<grid_for(n, EW_THREADS * EW_U, 8), EW_THREADS, 0, ctx->stream>>>(ip, k, perm, n, op);
    return launch_check("k_gather");
}

int canonicalize(tid_ctx *ctx, const int32_t *const *cols, int k, const int8_t *vars, int64_t n, bool dedupe,
                 const Bounds *bounds, tid_set **out, int sorted_tail) {
    *out = nullptr;
    tid_set *set = nullptr;
    TID_TRY(set_alloc(ctx, k, vars, n, &set));
    int rc = TID_OK;
    if (n == 0) {
        rc = set_rows_const(set, 0);
    } else {
        uint32_t hmin[TID_MAX_COLS], hmax[TID_MAX_COLS];
        if (bounds) {
            for (int c = 0; c < k; ++c) {
                hmin[c] = bounds->lo[c];
                hmax[c] = bounds->hi[c];
            }
        } else {
            rc = column_ranges(ctx, cols, k, n, hmin, hmax);
        }
        if (rc == TID_OK) {
            set->bounded = true;
            for (int c = 0; c < k; ++c) {
                set->lo[c] = hmin[c];
                set->hi[c] = hmax[c];
            }
        }
        int total = 0;
        PackSpec ps{};
        if (rc == TID_OK) {
            for (int c = k - 1; c >= 0; --c) {
                const int bits = range_bits(hmin[c], hmax[c]);
                ps.min[c] = hmin[c];
                ps.shift[c] = (uint32_t)total;
                ps.mask[c] = bits == 0 ? 0ull : ((1ull << bits) - 1ull);
                total += bits;
            }
        }
        // the trailing columns the rows are sorted by occupy the key bits below
        // the field of the last column before them
        const int sorted_bits = sorted_tail <= 0 ? 0 : (sorted_tail >= k ? total : (int)ps.shift[k - sorted_tail - 1]);
        if (rc == TID_OK && total <= 32) {
            rc = canonical_packed<uint32_t>(ctx, cols, k, n, dedupe, ps, total, sorted_bits, set);
        } else if (rc == TID_OK && total <= 64) {
            rc = canonical_packed<unsigned long long>(ctx, cols, k, n, dedupe, ps, total, sorted_bits, set);
        } else if (rc == TID_OK) {
            int32_t *perm = nullptr;
            rc = dev_alloc(ctx, (void **)&perm, (size_t)n * 4);
            if (rc == TID_OK) rc = sort_perm_ranges(ctx, cols, k, n, hmin, hmax, perm, sorted_tail);
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
    }
    if (rc == TID_OK) rc = set_ready(set);
    if (rc != TID_OK) {
        set_free(set);
        return rc;
    }
    *out = set;
    return TID_OK;
}

}  // namespace tid
