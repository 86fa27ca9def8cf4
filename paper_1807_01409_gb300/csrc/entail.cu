// tid_entail: RDFS entailment rules as two searches and a join (Section 5,
// Table "RDFS Entailment rules" and the Rule-11 walk-through).
//
//  1. search the schema premise (?a TERM ?b) -- K1 -- and extract its result
//     vector (a, b) -- K3/K4;
//  2. its distinct terms at the join position (the paper's keys of the second
//     GPUSearch) -- a projection with DISTINCT -- go into an open-addressing
//     table;
//  3. one pass over the store keeps the triples of the other premise whose term
//     at the join position is in the table (K3 with a hash probe per triple,
//     in store order) and extracts their variables;
//  4. the two result vectors are joined on the shared term (K5/K6) and the
//     conclusion's terms kept with DISTINCT.  When the conclusion is a pair of
//     terms, one from each premise, this is done without materialising the
//     join: each data row sets the bits of its pairs in a bit matrix indexed
//     by (rank of the schema term, data term - min), and the set bits, read
//     in order, are the distinct pairs already in canonical order.
#include <algorithm>
#include <vector>

#include "ops.cuh"

namespace tid {
int bind_set(tid_ctx *ctx, const tid_store *st, const tid_pattern &pat, const tid_set *idx, const tid_pred *preds,
             int n_preds, tid_set **out);
}  // namespace tid

using namespace tid;

namespace {

enum Term { NONE = -1, TYPE = 0, DOMAIN, RANGE, SUBPROP, SUBCLASS };

// variable ids used inside the evaluation (a and b of the schema premise, then
// the data premise's own variables)
constexpr int8_t VA = 10, VB = 11, VC = 12, VD = 13;

struct Rule {
    int schema;          // the schema premise is (?a schema ?b), a = VA, b = VB
    int8_t on;           // join variable: VA or VB
    int data_fixed;      // data premise: fixed predicate term, or NONE
    int key_slot;        // slot of the join variable in the data premise
    int8_t data_var[3];  // data premise variables per slot (-1: the fixed term or unused)
    int8_t then_var[3];  // conclusion per slot: a variable, or -1 for then_term
    int then_term;       // the conclusion's fixed predicate (slot 1), or NONE
};

bool rule_of(int id, Rule *r) {
    switch (id) {
        case TID_RULE_R2: *r = Rule{DOMAIN, VA, NONE, 1, {VC, VA, -1}, {VC, -1, VB}, TYPE}; return true;
        case TID_RULE_R3: *r = Rule{RANGE, VA, NONE, 1, {-1, VA, VC}, {VC, -1, VB}, TYPE}; return true;
        case TID_RULE_R5: *r = Rule{SUBPROP, VB, SUBPROP, 0, {VB, -1, VC}, {VA, -1, VC}, SUBPROP}; return true;
        case TID_RULE_R7: *r = Rule{SUBPROP, VA, NONE, 1, {VC, VA, VD}, {VC, VB, VD}, NONE}; return true;
        case TID_RULE_R9: *r = Rule{SUBCLASS, VA, TYPE, 2, {VC, -1, VA}, {VC, -1, VB}, TYPE}; return true;
        case TID_RULE_R11: *r = Rule{SUBCLASS, VB, SUBCLASS, 0, {VB, -1, VC}, {VA, -1, VC}, SUBCLASS}; return true;
        default: return false;
    }
}

__global__ void k_fill_i32(int32_t *__restrict__ out, int64_t n, int32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = v;
}

constexpr int BM_THREADS = 256;
constexpr uint32_t KEY_HASH = 0x9E3779B1u;      // multiplicative (Knuth) hash of the key table

__host__ __device__ __forceinline__ uint32_t home_slot(int32_t key, int tbits) {
    return ((uint32_t)key * KEY_HASH) >> (32 - tbits);
}

// slot of `key` in the open-addressing key table, or -1 (0 is the empty slot
// and never a key); at most one sweep of the table
__device__ __forceinline__ int find_slot(const int32_t *__restrict__ table, int tbits, int32_t key) {
    if (key == 0) return -1;
    const uint32_t mask = (1u << tbits) - 1u;
    uint32_t h = home_slot(key, tbits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const int32_t t = table[h];
        if (t == key) return (int)h;
        if (t == 0) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ uint32_t sort_order(int32_t x) { return (uint32_t)x ^ 0x80000000u; }

constexpr int BM_U = 4;  // rows per lane per step of the marking kernels (loads in flight)

// A warp's step: rows i0 + 32 u + lane, u < BM_U, i0 warp-uniform (so every
// lane takes part in the shuffles below).
__device__ __forceinline__ int64_t bm_first() {
    return (int64_t)blockIdx.x * (BM_THREADS * BM_U) + (int64_t)(threadIdx.x >> 5) * (32 * BM_U);
}
__device__ __forceinline__ int64_t bm_stride() { return (int64_t)gridDim.x * (BM_THREADS * BM_U); }

// flags gets one bit per table slot whose key occurs in key[0, n): the distinct
// join terms of the data premise's rows.  A lane skips a row whose slot equals
// the previous lane's, and sets a bit only while it is clear.  Bits collect in
// shared memory when SMEM, else in global memory directly.
template <bool SMEM>
__global__ void __launch_bounds__(BM_THREADS) k_mark_keys(const int32_t *__restrict__ key, int64_t n,
                                                          const int32_t *__restrict__ table, int tbits,
                                                          uint32_t *__restrict__ flags) {
    extern __shared__ uint32_t s_f[];
    const uint32_t words = ((1u << tbits) + 31u) >> 5;
    if (SMEM) {
        for (uint32_t w = threadIdx.x; w < words; w += BM_THREADS) s_f[w] = 0;
        __syncthreads();
    }
    volatile uint32_t *f = SMEM ? s_f : flags;
    const unsigned lane = threadIdx.x & 31;
    for (int64_t i0 = bm_first(); i0 < n; i0 += bm_stride()) {
        int32_t x[BM_U];
#pragma unroll
        for (int u = 0; u < BM_U; ++u) {
            const int64_t i = i0 + 32 * u + lane;
            x[u] = i < n ? key[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < BM_U; ++u) {
            const int h = find_slot(table, tbits, x[u]);
            const int hp = __shfl_up_sync(0xffffffffu, h, 1);
            if (h >= 0 && (lane == 0 || hp != h)) {
                const uint32_t b = 1u << (h & 31);
                if (!(f[h >> 5] & b)) atomicOr((uint32_t *)f + (h >> 5), b);
            }
        }
    }
    if (SMEM) {
        __syncthreads();
        for (uint32_t w = threadIdx.x; w < words; w += BM_THREADS)
            if (s_f[w]) atomicOr(flags + w, s_f[w]);
    }
}

// The conclusion's distinct pairs as the set bits of a matrix.  A data-premise
// row (join term, term t) joined with the schema rows of that join term gives
// the pairs (r, t) for A's other terms r.  r is ranked among A's distinct
// values of that term (ascending) and t is taken as d = order(t) - vmin.  Rows
// of the matrix follow the conclusion's first term and are 2^lg bits wide
// (the second term's span rounded up to a power of two): the pair is bit
// (r << lg) + d when A's term comes first, (d << lg) + r when t does.  The set
// bits in ascending order are the canonical distinct rows.
struct PairBits {
    const int32_t *key, *val;  // data-premise rows: join term, conclusion term
    int64_t n;
    const int32_t *table;  // the join terms (open addressing)
    int tbits;
    const uint32_t *off;    // slot h: A's ranks are rank[off[h] .. off[h + 1])
    const uint32_t *rank;
    const uint32_t *kmask;  // slot h: the same ranks as a mask (t first, 2^lg <= 32)
    uint32_t vmin;
    int lg;
    int a_first;
    uint32_t *bits;
};

// General form: one atomic OR per (row, rank) whose bit is not yet set; a
// lane skips a row equal, in slot and term, to the previous lane's.
__global__ void __launch_bounds__(BM_THREADS) k_pair_bits_list(PairBits P) {
    const unsigned lane = threadIdx.x & 31;
    for (int64_t i0 = bm_first(); i0 < P.n; i0 += bm_stride()) {
        int32_t x[BM_U], t[BM_U];
#pragma unroll
        for (int u = 0; u < BM_U; ++u) {
            const int64_t i = i0 + 32 * u + lane;
            x[u] = i < P.n ? P.key[i] : 0;
            t[u] = i < P.n ? P.val[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < BM_U; ++u) {
            const int h = find_slot(P.table, P.tbits, x[u]);
            const uint32_t d = sort_order(t[u]) - P.vmin;
            const int hp = __shfl_up_sync(0xffffffffu, h, 1);
            const uint32_t dp = __shfl_up_sync(0xffffffffu, d, 1);
            if (h < 0 || (lane > 0 && hp == h && dp == d)) continue;
            for (uint32_t j = P.off[h]; j < P.off[h + 1]; ++j) {
                const uint64_t r = P.rank[j];
                const uint64_t g = P.a_first ? (r << P.lg) + d : ((uint64_t)d << P.lg) + r;
                const uint32_t b = 1u << (g & 31);
                if (!(P.bits[g >> 5] & b)) atomicOr(P.bits + (g >> 5), b);  // read first, as above
            }
        }
    }
}

// t first and rows of at most 32 bits: a row's ranks are one mask within one
// word.  Lanes holding consecutive rows of the same word OR their masks (a
// segmented scan across the warp) and the last lane of each run writes it.
__global__ void __launch_bounds__(BM_THREADS) k_pair_bits_mask(PairBits P) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned le = lane == 31 ? 0xFFFFFFFFu : (2u << lane) - 1u;  // lanes <= this one
    for (int64_t i0 = bm_first(); i0 < P.n; i0 += bm_stride()) {
        int32_t x[BM_U], t[BM_U];
#pragma unroll
        for (int u = 0; u < BM_U; ++u) {
            const int64_t i = i0 + 32 * u + lane;
            x[u] = i < P.n ? P.key[i] : 0;
            t[u] = i < P.n ? P.val[i] : 0;
        }
#pragma unroll
        for (int u = 0; u < BM_U; ++u) {
            const int h = find_slot(P.table, P.tbits, x[u]);
            const uint64_t g = (uint64_t)(sort_order(t[u]) - P.vmin) << P.lg;
            const uint64_t word = h >= 0 ? g >> 5 : ~0ull;
            uint32_t acc = h >= 0 ? P.kmask[h] << (g & 31) : 0u;
            const uint64_t wp = __shfl_up_sync(0xffffffffu, word, 1);
            const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || wp != word);
            const int start = 31 - __clz(heads & le);
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, acc, d);
                if ((int)lane - d >= start) acc |= o;
            }
            const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
            // most rows repeat a pair already set: read before the atomic (a
            // stale read only costs the atomic)
            if (h >= 0 && tail && (P.bits[word] & acc) != acc) atomicOr(P.bits + word, acc);
        }
    }
}

// Reading the matrix out: segment s is words [s R 32, (s + 1) R 32), R rounds
// of 32 words, one warp per segment (a round's words one per lane).
__device__ __forceinline__ int64_t seg_of_warp() { return (int64_t)blockIdx.x * (BM_THREADS / 32) + (threadIdx.x >> 5); }

// counts[s] = set bits of segment s
__global__ void __launch_bounds__(BM_THREADS) k_seg_bits(const uint32_t *__restrict__ bits, int64_t nwords, int R,
                                                         int64_t nseg, uint32_t *__restrict__ counts) {
    const int64_t s = seg_of_warp();
    if (s >= nseg) return;
    const unsigned lane = threadIdx.x & 31;
    const int64_t w0 = s * R * 32 + lane;
    uint32_t c = 0;
#pragma unroll 8
    for (int r = 0; r < R; ++r) {
        const int64_t w = w0 + (int64_t)r * 32;
        c += w < nwords ? __popc(bits[w]) : 0u;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if (lane == 0) counts[s] = c;
}

// offs[s] = sum of counts[0, s) (64-bit), *total = sum of all.  One CTA steps
// through the counts 8192 at a time (eight consecutive ones per thread) with a
// carry.
__global__ void __launch_bounds__(1024) k_scan_segs(const uint32_t *__restrict__ counts, int64_t nseg,
                                                    unsigned long long *__restrict__ offs,
                                                    unsigned long long *__restrict__ total) {
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_chunk;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;
    for (int64_t base = 0; base < nseg; base += 1024 * 8) {
        const int64_t e0 = base + (int64_t)threadIdx.x * 8;
        uint32_t c[8];
        unsigned long long s = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            c[j] = e0 + j < nseg ? counts[e0 + j] : 0u;
            s += c[j];
        }
        unsigned long long x = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
            if ((int)lane >= d) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long v = s_w[lane];
            unsigned long long y = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long z = __shfl_up_sync(0xffffffffu, y, d);
                if ((int)lane >= d) y += z;
            }
            s_w[lane] = y - v;
            if (lane == 31) s_chunk = y;
        }
        __syncthreads();
        unsigned long long run = carry + s_w[warp] + x - s;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (e0 + j < nseg) offs[e0 + j] = run;
            run += c[j];
        }
        carry += s_chunk;
        __syncthreads();  // s_w and s_chunk are rewritten by the next chunk
    }
    if (threadIdx.x == 0) *total = carry;
}

struct PairOut {  // decoding a set bit into the conclusion's row
    const int32_t *rankval;  // A's distinct terms, ascending
    uint32_t vmin;
    int lg;
    int a_first;
    int32_t *out0, *out1;
    __device__ __forceinline__ void put(uint64_t g, uint64_t pos) const {
        const uint64_t hi = g >> lg, lo = g & ((1ull << lg) - 1ull);
        const uint64_t r = a_first ? hi : lo, d = a_first ? lo : hi;
        const int32_t a = rankval[r], t = (int32_t)((vmin + (uint32_t)d) ^ 0x80000000u);
        out0[pos] = a_first ? a : t;
        out1[pos] = a_first ? t : a;
    }
};

// The set bits of each segment, in order, as rows at the segment's offset.  A
// round whose words hold few bits (at most two each) is written lane by lane,
// the lanes' rows being consecutive; a denser round word by word, the word's
// bits one per lane, so the stores are coalesced either way.
__global__ void __launch_bounds__(BM_THREADS) k_emit_pairs(const uint32_t *__restrict__ bits, int64_t nwords, int R,
                                                           int64_t nseg, const unsigned long long *__restrict__ offs,
                                                           PairOut O) {
    const int64_t s = seg_of_warp();
    if (s >= nseg) return;
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t pos = offs[s];
    constexpr int AHEAD = 8;  // rounds whose words are loaded together
    for (int r0 = 0; r0 < R; r0 += AHEAD) {
        uint32_t va[AHEAD];
#pragma unroll
        for (int q = 0; q < AHEAD; ++q) {
            const int64_t w = (s * R + r0 + q) * 32 + lane;
            va[q] = r0 + q < R && w < nwords ? bits[w] : 0u;
        }
#pragma unroll
        for (int q = 0; q < AHEAD; ++q) {
            const int64_t wb = (s * R + r0 + q) * 32;  // the round's first word
            if (r0 + q >= R || wb >= nwords) break;
            const int64_t w = wb + lane;
            uint32_t v = va[q];
            const uint32_t c = __popc(v);
            uint32_t x = c;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
                if ((int)lane >= d) x += y;
            }
            const uint64_t mine = pos + x - c;
            const uint32_t tot = __shfl_sync(0xffffffffu, x, 31);
            if (__any_sync(0xffffffffu, c > 2)) {
                unsigned nz = __ballot_sync(0xffffffffu, v != 0);
                while (nz) {
                    const int L = __ffs(nz) - 1;
                    nz &= nz - 1;
                    const uint32_t wv = __shfl_sync(0xffffffffu, v, L);
                    const uint64_t b0 = __shfl_sync(0xffffffffu, mine, L);
                    if ((wv >> lane) & 1u) O.put((uint64_t)(wb + L) * 32 + lane, b0 + __popc(wv & lt));
                }
            } else {
                uint64_t at = mine;
                while (v) {
                    const int b = __ffs(v) - 1;
                    v &= v - 1;
                    O.put((uint64_t)w * 32 + b, at++);
                }
            }
            pos += tot;
        }
    }
}

// *count = set bits of words[0, n) (one CTA)
__global__ void __launch_bounds__(1024) k_count_bits(const uint32_t *__restrict__ words, int64_t n,
                                                     unsigned long long *__restrict__ count) {
    __shared__ unsigned long long s_w[32];
    unsigned long long c = 0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) c += (unsigned)__popc(words[i]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        c = s_w[threadIdx.x];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (threadIdx.x == 0) *count = c;
    }
}

// mm[0] = min, mm[1] = max of col[0, n) in sort order (mm preset to ~0, 0)
__global__ void k_col_range(const int32_t *__restrict__ col, int64_t n, uint32_t *__restrict__ mm) {
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = sort_order(col[i]);
        lo = min(lo, v);
        hi = max(hi, v);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    }
    if ((threadIdx.x & 31) == 0) {  // skip an atomic that cannot tighten the bound
        if (lo < __ldcg(mm)) atomicMin(mm, lo);
        if (hi > __ldcg(mm + 1)) atomicMax(mm + 1, hi);
    }
}

struct Sets {  // frees what it holds
    std::vector<tid_set *> v;
    ~Sets() {
        for (tid_set *s : v) set_free(s);
    }
    tid_set *keep(tid_set *s) {
        v.push_back(s);
        return s;
    }
};

int rows_of(tid_set *s, int64_t *n) { return set_rows_host(s, n); }

struct Buf {  // a device allocation freed on scope exit
    tid_ctx *c;
    void *p = nullptr;
    ~Buf() {
        if (p) dev_free(c, p);
    }
};

constexpr int64_t PAIR_MAX_SCHEMA_ROWS = 1 << 22;  // schema rows ranked on the host
// A matrix of up to 64 MiB stays mostly in L2 and is always taken; a larger
// one only up to 4 bytes per data-premise row: beyond L2 every pair's bit is a
// random DRAM read-modify-write, and joining and sorting the rows costs less
// (R9 at 200M: a 1.28 GB matrix took 4.8 ms to fill and read out).
constexpr uint64_t PAIR_MIN_BYTES = 64ull << 20;
constexpr uint64_t PAIR_BYTES_PER_ROW = 4;
constexpr uint64_t PAIR_MAX_BYTES = 4ull << 30;

// The conclusion as the bit matrix of its distinct pairs (PairBits), when it
// has two terms, A's non-join term and one of the data premise's, and the
// matrix is small enough.  *out stays null when this form does not apply and
// the join is taken instead.
//   A: the schema premise's rows (join term and other term); B: the data
//   premise's rows (nb), its column tcol the conclusion's term; table/d_table:
//   the key table on the host and the device.
int conclude_pairs(tid_ctx *ctx, const Rule &R, tid_set *A, tid_set *B, int64_t nb, const int8_t *bvars, int kb,
                   const std::vector<int32_t> &table, const int32_t *d_table, int tbits, const int8_t *cvars,
                   int kc, tid_set **out) {
    *out = nullptr;
    if (kc != 2 || nb == 0) return TID_OK;
    const int8_t other = R.on == VA ? VB : VA;  // A's term that is not the join term
    const int a_pos = cvars[0] == other ? 0 : (cvars[1] == other ? 1 : -1);
    if (a_pos < 0) return TID_OK;
    const int8_t tv = cvars[1 - a_pos];
    int tcol = -1, kcol = -1;
    for (int c = 0; c < kb; ++c) {
        if (bvars[c] == tv && tv != R.on) tcol = c;
        if (bvars[c] == R.on) kcol = c;
    }
    int ak = -1, ao = -1;
    for (int c = 0; c < A->k; ++c) {
        if (A->vars[c] == R.on) ak = c;
        if (A->vars[c] == other) ao = c;
    }
    int64_t nA = 0;
    TID_TRY(set_rows_host(A, &nA));
    if (tcol < 0 || kcol < 0 || ak < 0 || ao < 0 || nA == 0 || nA > PAIR_MAX_SCHEMA_ROWS) return TID_OK;
    cudaStream_t stream = ctx->stream;

    // the range of the data premise's term, and A's rows on the host
    Buf rb{ctx};
    TID_TRY(dev_alloc(ctx, &rb.p, 2 * sizeof(uint32_t)));
    uint32_t *mm = (uint32_t *)rb.p;
    TID_TRY_CUDA(cudaMemsetAsync(mm, 0xFF, sizeof(uint32_t), stream), "range");
    TID_TRY_CUDA(cudaMemsetAsync(mm + 1, 0, sizeof(uint32_t), stream), "range");
    k_col_range<<<grid_for(nb, 256, 8), 256, 0, stream>>>(B->col[tcol], nb, mm);
    TID_TRY(launch_check("k_col_range"));
    uint32_t hmm[2] = {0, 0};
    TID_TRY_CUDA(cudaMemcpyAsync(hmm, mm, sizeof hmm, cudaMemcpyDeviceToHost, stream), "range");
    std::vector<int32_t> arows((size_t)nA * A->k);
    int64_t got = 0;
    TID_TRY(tid_set_to_host(A, arows.data(), nA, &got));  // synchronises
    if (hmm[0] > hmm[1]) return TID_OK;

    // A's other terms ranked; the matrix's size decides the form
    std::vector<int32_t> vals((size_t)nA);
    for (int64_t i = 0; i < nA; ++i) vals[(size_t)i] = arows[(size_t)i * A->k + ao];
    std::sort(vals.begin(), vals.end());
    vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
    const uint64_t na = vals.size(), w = (uint64_t)(hmm[1] - hmm[0]) + 1;
    const uint64_t nrows = a_pos == 0 ? na : w, width = a_pos == 0 ? w : na;  // matrix rows, bits per row
    int lg = 0;
    while ((1ull << lg) < width) ++lg;
    int lr = 0;
    while ((1ull << lr) < nrows) ++lr;
    if (lg + lr > 40) return TID_OK;  // far beyond the size limit below
    const uint64_t nwords = ((nrows << lg) + 31) / 32, bytes = nwords * sizeof(uint32_t);
    if (bytes > std::max(PAIR_MIN_BYTES, PAIR_BYTES_PER_ROW * (uint64_t)nb) || bytes > PAIR_MAX_BYTES) return TID_OK;

    // per key slot, the ranks of its schema rows' other terms (ascending)
    const uint32_t tsize = 1u << tbits;
    std::vector<std::pair<uint32_t, uint32_t>> hr;
    hr.reserve((size_t)nA);
    for (int64_t i = 0; i < nA; ++i) {
        const int32_t key = arows[(size_t)i * A->k + ak];
        if (key == 0) continue;  // 0 never joins
        uint32_t h = home_slot(key, tbits);
        for (uint32_t probe = 0; probe < tsize && table[h] != key; ++probe) h = (h + 1) & (tsize - 1);
        if (table[h] != key) continue;
        const int32_t v = arows[(size_t)i * A->k + ao];
        hr.emplace_back(h, (uint32_t)(std::lower_bound(vals.begin(), vals.end(), v) - vals.begin()));
    }
    std::sort(hr.begin(), hr.end());
    hr.erase(std::unique(hr.begin(), hr.end()), hr.end());
    const bool use_mask = a_pos == 1 && lg <= 5;  // a row's ranks fit one word
    // layout: rank values (na) | off (tsize + 1) | ranks | masks (tsize, when used)
    std::vector<uint32_t> meta(na + tsize + 1 + hr.size() + (use_mask ? tsize : 0), 0u);
    uint32_t *m_off = meta.data() + na, *m_rank = m_off + tsize + 1, *m_mask = m_rank + hr.size();
    for (uint64_t r = 0; r < na; ++r) meta[r] = (uint32_t)vals[r];
    for (size_t j = 0; j < hr.size(); ++j) {
        m_off[hr[j].first + 1]++;
        m_rank[j] = hr[j].second;
        if (use_mask) m_mask[hr[j].first] |= 1u << hr[j].second;
    }
    for (uint32_t h = 0; h < tsize; ++h) m_off[h + 1] += m_off[h];
    Buf mb{ctx};
    TID_TRY(dev_alloc(ctx, &mb.p, meta.size() * sizeof(uint32_t)));
    TID_TRY_CUDA(cudaMemcpyAsync(mb.p, meta.data(), meta.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, stream),
                 "pair ranks");
    const uint32_t *d_meta = (const uint32_t *)mb.p;

    // the matrix's bits, then its set bits in order as rows
    Buf bb{ctx};
    TID_TRY(dev_alloc(ctx, &bb.p, bytes));
    uint32_t *bits = (uint32_t *)bb.p;
    TID_TRY_CUDA(cudaMemsetAsync(bits, 0, bytes, stream), "pair bits");
    const PairBits P{B->col[kcol], B->col[tcol], nb, d_table, tbits,
                     d_meta + na, d_meta + na + tsize + 1, use_mask ? d_meta + na + tsize + 1 + hr.size() : nullptr,
                     hmm[0], lg, a_pos == 0 ? 1 : 0, bits};
    const unsigned grid = grid_for(nb, BM_THREADS * BM_U, 8);
    if (use_mask) {
        k_pair_bits_mask<<<grid, BM_THREADS, 0, stream>>>(P);
        TID_TRY(launch_check("k_pair_bits_mask"));
    } else {
        k_pair_bits_list<<<grid, BM_THREADS, 0, stream>>>(P);
        TID_TRY(launch_check("k_pair_bits_list"));
    }
    // segments of R rounds of 32 words, at most 2^16 of them (one warp each)
    const int rounds = (int)std::max<int64_t>(8, ceil_div((int64_t)nwords, (int64_t)32 << 16));
    const int64_t nseg = ceil_div((int64_t)nwords, (int64_t)rounds * 32);
    const unsigned seg_ctas = (unsigned)ceil_div(nseg, BM_THREADS / 32);
    const int64_t cpad = (nseg + 1) & ~(int64_t)1;
    Buf sb{ctx};
    TID_TRY(dev_alloc(ctx, &sb.p, sizeof(uint32_t) * cpad + sizeof(unsigned long long) * (nseg + 1)));
    uint32_t *counts = (uint32_t *)sb.p;
    unsigned long long *offs = (unsigned long long *)(counts + cpad), *d_total = offs + nseg;
    k_seg_bits<<<seg_ctas, BM_THREADS, 0, stream>>>(bits, (int64_t)nwords, rounds, nseg, counts);
    TID_TRY(launch_check("k_seg_bits"));
    k_scan_segs<<<1, 1024, 0, stream>>>(counts, nseg, offs, d_total);
    TID_TRY(launch_check("k_scan_segs"));
    unsigned long long total = 0;
    TID_TRY_CUDA(cudaMemcpyAsync(&total, d_total, sizeof total, cudaMemcpyDeviceToHost, stream), "pair rows");
    TID_TRY_CUDA(cudaStreamSynchronize(stream), "pair rows");
    tid_set *C = nullptr;
    TID_TRY(set_alloc(ctx, 2, cvars, (int64_t)total, &C));
    int rc = TID_OK;
    if (total > 0) {
        const PairOut O{(const int32_t *)d_meta, hmm[0], lg, a_pos == 0 ? 1 : 0, C->col[0], C->col[1]};
        k_emit_pairs<<<seg_ctas, BM_THREADS, 0, stream>>>(bits, (int64_t)nwords, rounds, nseg, offs, O);
        rc = launch_check("k_emit_pairs");
    }
    if (rc == TID_OK) rc = set_rows_const(C, (int64_t)total);
    if (rc == TID_OK) {
        // valid bounds (sort order) of each column
        const uint32_t alo = (uint32_t)vals.front() ^ 0x80000000u, ahi = (uint32_t)vals.back() ^ 0x80000000u;
        C->bounded = true;
        C->lo[a_pos] = alo;
        C->hi[a_pos] = ahi;
        C->lo[1 - a_pos] = hmm[0];
        C->hi[1 - a_pos] = hmm[1];
        rc = set_ready(C);
    }
    if (rc != TID_OK) {
        set_free(C);
        return rc;
    }
    *out = C;
    return TID_OK;
}

}  // namespace

extern "C" int tid_entail(tid_ctx *ctx, const tid_store *st, int rule, const tid_rdfs_vocab *vocab, tid_set **out,
                          tid_entail_stats *stats) {
    clear_error();
    tid::Range nvtx_range("tid_entail");
    if (!ctx || !st || !vocab || !out) return fail(TID_ERR_ARG, "tid_entail: null argument");
    *out = nullptr;
    if (st->ctx != ctx) return fail(TID_ERR_ARG, "tid_entail: store belongs to another context");
    Rule R;
    if (!rule_of(rule, &R)) return fail(TID_ERR_ARG, "tid_entail: unknown rule %d", rule);
    const int32_t term[5] = {vocab->type, vocab->domain, vocab->range, vocab->sub_property_of, vocab->sub_class_of};
    for (int t = 0; t < 5; ++t)
        if (term[t] <= 0) return fail(TID_ERR_ID, "tid_entail: vocabulary ID %d is not positive", term[t]);
    DeviceGuard g(ctx->device);
    cudaStream_t stream = ctx->stream;
    tid_entail_stats sx{};
    Sets hold;

    // 1) schema premise (?a TERM ?b) -> (a, b)
    tid_pattern sp{};
    sp.p = term[R.schema];
    sp.var[0] = VA;
    sp.var[1] = -1;
    sp.var[2] = VB;
    tid_set *idx1 = nullptr, *A = nullptr;
    TID_TRY(tid_match(ctx, st, sp, &idx1));
    hold.keep(idx1);
    TID_TRY(rows_of(idx1, &sx.res1));
    TID_TRY(bind_set(ctx, st, sp, idx1, nullptr, 0, &A));
    hold.keep(A);

    // 2) its distinct join terms -> key table
    tid_set *K = nullptr;
    TID_TRY(project_set(ctx, A, &R.on, 1, &K));
    hold.keep(K);
    TID_TRY(rows_of(K, &sx.dist1));
    std::vector<int32_t> keys((size_t)sx.dist1);
    if (sx.dist1 > 0) {
        int64_t got = 0;
        TID_TRY(tid_set_to_host(K, keys.data(), sx.dist1, &got));
    }
    // open addressing, at most half full; the home slot is the top bits of a
    // multiplicative hash (Knuth), which depend on every bit of the key
    int tbits = 4;
    while ((1ull << tbits) < 2 * (uint64_t)std::max<int64_t>(sx.dist1, 1)) ++tbits;
    const uint32_t tsize = 1u << tbits;
    std::vector<int32_t> table(tsize, 0);
    for (int32_t key : keys) {  // keys are distinct and positive (0 never joins)
        if (key == 0) continue;
        uint32_t h = home_slot(key, tbits);
        while (table[h] != 0) h = (h + 1) & (tsize - 1);
        table[h] = key;
    }
    void *d_table = nullptr;
    TID_TRY(dev_alloc(ctx, &d_table, sizeof(int32_t) * tsize));
    struct TableFree {
        tid_ctx *c;
        void *p;
        ~TableFree() { dev_free(c, p); }
    } tf{ctx, d_table};
    TID_TRY_CUDA(cudaMemcpyAsync(d_table, table.data(), sizeof(int32_t) * tsize, cudaMemcpyHostToDevice, stream),
                 "key table");

    // 3) the data premise's triples whose join term is a key, in store order
    int8_t bvars[3], bsrc[3];
    int kb = 0;
    for (int slot = 0; slot < 3; ++slot) {
        const int8_t v = R.data_var[slot];
        if (v < 0) continue;
        bool seen = false;
        for (int c = 0; c < kb; ++c) seen = seen || bvars[c] == v;
        if (!seen) {
            bvars[kb] = v;
            bsrc[kb] = (int8_t)slot;
            ++kb;
        }
    }
    tid_set *Braw = nullptr, *B = nullptr;
    TID_TRY(set_alloc(ctx, kb, bvars, st->n, &Braw));
    hold.keep(Braw);
    const int fixed_slot = R.data_fixed == NONE ? -1 : 1;
    const int32_t fixed_val = R.data_fixed == NONE ? 0 : term[R.data_fixed];
    if (sx.dist1 > 0) {
        TID_TRY(compact_semijoin(ctx, st, fixed_slot, fixed_val, R.key_slot, (const int32_t *)d_table, tbits,
                                 bsrc, Braw));
    } else {
        TID_TRY(set_rows_const(Braw, 0));
    }
    TID_TRY(set_ready(Braw));
    TID_TRY(rows_of(Braw, &sx.res2));
    // the distinct join terms among them (the paper's #Dist2): the rows mark
    // their term's slot of the key table, and the marks are counted
    int kcol = 0;
    for (int c = 0; c < kb; ++c)
        if (bvars[c] == R.on) kcol = c;
    {
        const uint32_t fwords = (tsize + 31) / 32, fpad = (fwords + 1) & ~1u;
        Buf fb{ctx};
        TID_TRY(dev_alloc(ctx, &fb.p, sizeof(uint32_t) * fpad + sizeof(unsigned long long)));
        uint32_t *flags = (uint32_t *)fb.p;
        unsigned long long *d_cnt = (unsigned long long *)(flags + fpad);
        TID_TRY_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t) * fwords, stream), "key marks");
        if (sx.res2 > 0) {
            const unsigned grid = grid_for(sx.res2, BM_THREADS * BM_U, 8);
            const size_t fsmem = sizeof(uint32_t) * fwords;
            if (fsmem <= 32 * 1024)
                k_mark_keys<true><<<grid, BM_THREADS, fsmem, stream>>>(Braw->col[kcol], sx.res2,
                                                                       (const int32_t *)d_table, tbits, flags);
            else
                k_mark_keys<false><<<grid, BM_THREADS, 0, stream>>>(Braw->col[kcol], sx.res2,
                                                                    (const int32_t *)d_table, tbits, flags);
            TID_TRY(launch_check("k_mark_keys"));
        }
        k_count_bits<<<1, 1024, 0, stream>>>(flags, fwords, d_cnt);
        TID_TRY(launch_check("k_count_bits"));
        unsigned long long cnt = 0;
        TID_TRY_CUDA(cudaMemcpyAsync(&cnt, d_cnt, sizeof cnt, cudaMemcpyDeviceToHost, stream), "key count");
        TID_TRY_CUDA(cudaStreamSynchronize(stream), "key count");
        sx.dist2 = (int64_t)cnt;
    }
    B = Braw;  // rows in store order: neither form of step 4 needs an order

    // 4) the join on the shared term, the conclusion's terms kept with
    //    DISTINCT.  A two-term conclusion with one term from each premise is
    //    the bit matrix of its distinct pairs, when that is small enough;
    //    otherwise the join is a hash join with the schema side (the small one)
    //    as the table, its rows left in the order written, and the conclusion's
    //    terms are put in canonical order with DISTINCT -- the one sort of the
    //    rule.
    int8_t cvars[3];
    int kc = 0;
    for (int slot = 0; slot < 3; ++slot)
        if (R.then_var[slot] >= 0) cvars[kc++] = R.then_var[slot];
    tid_set *C = nullptr;
    TID_TRY(conclude_pairs(ctx, R, A, B, sx.res2, bvars, kb, table, (const int32_t *)d_table, tbits, cvars, kc,
                           &C));
    if (C) {
        hold.keep(C);
    } else {
        tid_set *J = nullptr;
        TID_TRY(join_sets(ctx, A, B, TID_JOIN_HASH, &J, false));
        hold.keep(J);
        const int32_t *ccols[3];
        Bounds cb{};
        for (int i = 0; i < kc; ++i) {
            int c = 0;
            while (J->vars[c] != cvars[i]) ++c;
            ccols[i] = J->col[c];
            cb.lo[i] = J->lo[c];
            cb.hi[i] = J->hi[c];
        }
        int64_t nj = 0;
        TID_TRY(rows_of(J, &nj));
        TID_TRY(canonicalize(ctx, ccols, kc, cvars, nj, true, J->bounded ? &cb : nullptr, &C));
        hold.keep(C);
    }
    int64_t rows = 0;
    TID_TRY(rows_of(C, &rows));

    // the (s, p, o) set: C's columns, the fixed predicate in the middle when the
    // conclusion has one (a constant column keeps C's order canonical)
    const int8_t ovars[3] = {0, 1, 2};
    tid_set *O = nullptr;
    TID_TRY(set_alloc(ctx, 3, ovars, rows, &O));
    int rc = TID_OK;
    int c = 0;
    for (int slot = 0; slot < 3 && rc == TID_OK; ++slot) {
        if (R.then_var[slot] >= 0) {
            if (rows > 0) {
                cudaError_t e = cudaMemcpyAsync(O->col[slot], C->col[c], (size_t)rows * 4, cudaMemcpyDeviceToDevice,
                                                stream);
                if (e != cudaSuccess) rc = fail_cuda(e, "conclusion column");
            }
            O->lo[slot] = C->lo[c];
            O->hi[slot] = C->hi[c];
            ++c;
        } else {
            const int32_t v = term[R.then_term];
            if (rows > 0) {
                k_fill_i32<<<grid_for(rows, 256, 8), 256, 0, stream>>>(O->col[slot], rows, v);
                rc = launch_check("k_fill_i32");
            }
            O->lo[slot] = O->hi[slot] = (uint32_t)v ^ 0x80000000u;
        }
    }
    O->bounded = C->bounded;
    if (rc == TID_OK) rc = set_rows_const(O, rows);
    if (rc == TID_OK) rc = set_ready(O);
    if (rc != TID_OK) {
        set_free(O);
        return rc;
    }
    sx.all = rows;
    if (stats) *stats = sx;
    *out = O;
    return TID_OK;
}
