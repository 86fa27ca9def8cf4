// Device side of the single-pass tile prefix (decoupled look-back).
//
// A kernel that compacts in one pass gives every CTA a tile number from a
// ticket counter (so tiles start in order and every predecessor of a tile is
// already running), lets warp 0 publish the tile's count, and then walks
// back over predecessors' status words until it meets an inclusive prefix.
// Every wait is bounded: after LB_SPIN_LIMIT polls the tile marks itself
// "gave up", sets TID_ERR_TIMEOUT in the error word and returns -1; a tile
// that sees a predecessor that gave up gives up at once.
#pragma once

#include "tid_internal.cuh"

namespace tid {

__device__ __forceinline__ unsigned long long lb_load(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void lb_store(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long lb_word(unsigned epoch, unsigned flag, unsigned value) {
    return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | value;
}

// Called by thread 0: draws this CTA's tile number.  Returns num_tiles (an
// invalid tile) if the counter was not at 0 when the launch began.
__device__ __forceinline__ unsigned lb_ticket(const Lookback &lb) {
    unsigned t = atomicAdd(lb.ticket, 1u);
    if (t == lb.num_tiles - 1) atomicExch(lb.ticket, 0u);
    if (t >= lb.num_tiles) {
        atomicExch(lb.err, TID_ERR_CUDA);
        return lb.num_tiles;
    }
    return t;
}

// Persistent kernels: every CTA draws tickets until it gets one >= num_tiles,
// so one launch draws exactly num_tiles + grid tickets; the last draw resets
// the counter.  Called by thread 0.
__device__ __forceinline__ unsigned lb_ticket_persistent(const Lookback &lb, unsigned grid) {
    unsigned t = atomicAdd(lb.ticket, 1u);
    if (t == lb.num_tiles + grid - 1) atomicExch(lb.ticket, 0u);
    return t;
}

// Mark a tile as given up without waiting (its CTA already gave up once).
__device__ __forceinline__ void lb_abort(const Lookback &lb, unsigned tile) {
    if ((threadIdx.x & 31) == 0) lb_store(lb.status + tile, lb_word(lb.epoch, LB_FLAG_ABORT, 0));
}

// Called by all 32 lanes of ONE warp.  Publishes `total` for `tile` and
// returns the tile's exclusive prefix (sum of the totals of tiles < tile), or
// -1 if a wait gave up.  Each lane reads LB_DEPTH consecutive predecessors, so
// one round trip to L2 inspects a window of 32 * LB_DEPTH tiles.
constexpr int LB_DEPTH = 8;

__device__ __forceinline__ long long lb_exclusive_prefix(const Lookback &lb, unsigned tile,
                                                         unsigned total) {
    const unsigned lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) lb_store(lb.status, lb_word(lb.epoch, LB_FLAG_PREFIX, total));
        return 0;
    }
    if (lane == 0) lb_store(lb.status + tile, lb_word(lb.epoch, LB_FLAG_AGG, total));
    long long excl = 0;
    long long pos = (long long)tile - 1;
    unsigned polls = 0;
    bool gave_up = false;
    while (true) {
        unsigned long long w[LB_DEPTH];
#pragma unroll
        for (int i = 0; i < LB_DEPTH; ++i) {
            const long long idx = pos - (long long)(lane * LB_DEPTH + i);
            w[i] = idx >= 0 ? lb_load(lb.status + idx) : lb_word(lb.epoch, LB_FLAG_PREFIX, 0);
        }
        // nearest-first scan of this lane's entries up to (and with) its first prefix
        bool has_pref = false, notready = false, aborted = false;
        unsigned long long sum = 0;
#pragma unroll
        for (int i = 0; i < LB_DEPTH; ++i) {
            if (has_pref) continue;
            const unsigned f = ((unsigned)(w[i] >> 34) == lb.epoch) ? (unsigned)(w[i] >> 32) & 3u : 0u;
            notready = notready || f == 0;
            aborted = aborted || f == LB_FLAG_ABORT;
            sum += (unsigned)w[i];
            has_pref = f == LB_FLAG_PREFIX;
        }
        const unsigned pref = __ballot_sync(0xffffffffu, has_pref);
        const unsigned nr = __ballot_sync(0xffffffffu, notready);
        const unsigned ab = __ballot_sync(0xffffffffu, aborted);
        const int stop = pref ? __ffs(pref) - 1 : 31;
        const unsigned upto = stop == 31 ? 0xffffffffu : ((2u << stop) - 1u);
        if (ab & upto) { gave_up = true; break; }
        if (nr & upto) {
            if (++polls > LB_SPIN_LIMIT) {
                if (lane == 0) atomicExch(lb.err, TID_ERR_TIMEOUT);
                gave_up = true;
                break;
            }
            __nanosleep(polls < 64 ? 32 : 256);
            continue;
        }
        unsigned long long v = (int)lane <= stop ? sum : 0ull;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        excl += (long long)v;
        if (pref) break;
        pos -= 32 * LB_DEPTH;
    }
    if (gave_up) {
        if (lane == 0) lb_store(lb.status + tile, lb_word(lb.epoch, LB_FLAG_ABORT, 0));
        return -1;
    }
    if (lane == 0)
        lb_store(lb.status + tile, lb_word(lb.epoch, LB_FLAG_PREFIX, (unsigned)(excl + total)));
    return excl;
}

// ---- grid barrier (cooperative launches only: every CTA is resident) --------

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All CTAs of a cooperative launch meet here; false if the wait gave up.
__device__ __forceinline__ bool grid_barrier(unsigned *counter, unsigned expected, int *err,
                                             unsigned limit = LB_SPIN_LIMIT) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1u);
        int ok = 1;
        unsigned polls = 0;
        while (ld_acquire_u32(counter) < expected) {
            if (++polls > limit) {
                atomicExch(err, TID_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace tid
