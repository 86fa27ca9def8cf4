// Internal declarations shared by the libtid translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "tid.h"

namespace tid {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
int fail(int code, const char *fmt, ...);
int fail_cuda(cudaError_t e, const char *what);
void clear_error();
// TID_OK if `device` is this process's GPU (the first device any call used),
// else TID_ERR_ARG
int claim_device(int device);

#define TID_TRY_CUDA(expr, what)                                   \
    do {                                                           \
        cudaError_t e_ = (expr);                                   \
        if (e_ != cudaSuccess) return ::tid::fail_cuda(e_, what);  \
    } while (0)

#define TID_TRY(expr)                   \
    do {                                \
        int rc_ = (expr);               \
        if (rc_ != TID_OK) return rc_;  \
    } while (0)

// ---------------------------------------------------------------------------
// single-pass look-back scratch (decoupled look-back prefix over tiles)
//
// One 64-bit status word per tile: [63:34] launch epoch, [33:32] flag,
// [31:0] value.  Flags: 1 = tile aggregate ready, 2 = inclusive prefix ready,
// 3 = tile gave up (a bounded wait ran out).  A word from an older launch has
// a different epoch and reads as "not ready", so the array is never cleared
// between launches.  Tile numbers come from a ticket counter; the CTA that
// draws the last ticket of a launch resets it to 0.
// ---------------------------------------------------------------------------
struct Lookback {
    unsigned long long *status;  // >= num_tiles words
    unsigned int *ticket;        // one counter, 0 between launches
    unsigned int epoch;          // 1 .. 2^30-1
    unsigned int num_tiles;
    int *err;                    // device-visible error word (TID_ERR_*)
};

// Where look-back scratch lives: `cap` status words, a ticket counter, the
// error word, and the host-side epoch counter advanced by every launch.
struct LbScratch {
    unsigned long long *status;
    size_t cap;
    unsigned int *ticket;
    int *err;
    unsigned int *epoch;
};

constexpr unsigned LB_FLAG_AGG = 1, LB_FLAG_PREFIX = 2, LB_FLAG_ABORT = 3;
constexpr unsigned LB_SPIN_LIMIT = 1u << 21;  // polls before a wait gives up

// ---------------------------------------------------------------------------
// objects behind the opaque handles
// ---------------------------------------------------------------------------
struct Slot {  // one int64 in mapped pinned host memory
    int64_t *host = nullptr;
    int64_t *dev = nullptr;
    int slab = -1, index = -1;
};

struct PendingSlot {  // a freed set's slot, reusable once its producer event completed
    Slot slot;
    cudaEvent_t ev;
};

struct SharedBlock {  // device allocations shared by several sets (freed with the last)
    void *ptr[2] = {nullptr, nullptr};
    int refs = 0;
};

}  // namespace tid

struct tid_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    // look-back scratch
    unsigned long long *lb_status = nullptr;
    size_t lb_cap = 0;           // status words allocated
    unsigned int *lb_ticket = nullptr;
    unsigned int epoch = 0;
    // error word in mapped pinned memory (written by kernels, read by host)
    int *err_host = nullptr;
    int *err_dev = nullptr;
    // mapped pinned slabs for row counts
    std::vector<int64_t *> slabs_host;
    std::vector<int64_t *> slabs_dev;
    std::vector<std::pair<int, int>> free_slots;
    std::vector<tid::PendingSlot> pending;
    std::mutex mu;
    // the batched search's last plan on this context (tid_batch_tuning)
    int batch_shape = -1, batch_keys = 0, batch_subs = 0;
    // testing aid (tid_ctx_inject_alloc_failure): allocations left before they fail
    std::atomic<int64_t> fail_after{-1};
    std::atomic<int64_t> allocs{0};
};

struct tid_store {
    tid_ctx *ctx = nullptr;
    int64_t n = 0;
    const int32_t *s = nullptr, *p = nullptr, *o = nullptr;
    void *owned = nullptr;  // single allocation holding the three columns, or null
    bool aligned16 = false; // all three columns 16-byte aligned
    // Whether the triples are in (s, p, o) order (int32 order, repeats
    // allowed): *d_unsorted is set at load by a check kernel when some triple
    // follows a larger one; `spo_sorted` caches it on the host once read
    // (-1: not read yet).
    int32_t *d_unsorted = nullptr;
    mutable int spo_sorted = -1;
};

struct tid_set {
    tid_ctx *ctx = nullptr;
    int k = 0;
    int8_t vars[TID_MAX_COLS] = {0};
    int64_t cap = 0;
    int32_t *col[TID_MAX_COLS] = {nullptr};
    int64_t *d_rows = nullptr;   // device row count
    tid::Slot slot;              // host mirror of the row count
    cudaEvent_t ready = nullptr; // recorded after the producing work
    int64_t rows_known = -1;
    void *block = nullptr;       // allocation holding the columns and d_rows
    tid::SharedBlock *shared = nullptr;  // or: a view into allocations shared with other sets
    // Valid bounds of each column's values in sort order (int32 ^ 0x80000000),
    // when known: lo[c] <= every value of column c <= hi[c].
    bool bounded = false;
    uint32_t lo[TID_MAX_COLS] = {0}, hi[TID_MAX_COLS] = {0};
};

namespace tid {

// device / context helpers (api.cu)
// An NVTX range over one C-ABI call (visible in profiler timelines; free when
// no tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};
int dev_alloc(tid_ctx *ctx, void **p, size_t bytes);
void dev_free(tid_ctx *ctx, void *p);
int lookback_scratch(tid_ctx *ctx, unsigned int num_tiles, Lookback *lb);
int ctx_scratch(tid_ctx *ctx, size_t words, LbScratch *sc);    // the context's scratch, >= words
int make_lookback(const LbScratch &sc, unsigned int num_tiles, Lookback *lb);  // next epoch
int set_alloc(tid_ctx *ctx, int k, const int8_t *vars, int64_t cap, tid_set **out);
int set_ready(tid_set *set);      // record the producer event
void set_free(tid_set *set);      // tid_set_free without clearing the error message
// A one-column set labelled -1 viewing `col` (rows known on the host, count in
// *d_rows on the device) inside sb's allocations; takes one reference on sb.
int set_view(tid_ctx *ctx, tid::SharedBlock *sb, int32_t *col, int64_t *d_rows, int64_t rows, tid_set **out);
int check_ctx_error(tid_ctx *ctx); // reads and clears the kernel error word
bool store_spo_sorted(const tid_store *st);  // triples in (s, p, o) order (waits for the load's check)
int launch_check(const char *what);

// kernels (match.cu)
int launch_match(cudaStream_t stream, const int32_t *S, const int32_t *P, const int32_t *O,
                 int64_t n, bool aligned16, int32_t ks, int32_t kp, int32_t ko,
                 int32_t *out, int64_t cap, int64_t *d_rows, int64_t *h_rows_dev,
                 const LbScratch &sc);
unsigned int match_scratch_words();  // status words one K1 launch may need

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int sm_count();  // SMs of the current device (queried once per device)

// Grid of a grid-stride kernel: one CTA per `per_cta` items, at most `per_sm`
// CTAs per SM, at least one.
inline unsigned grid_for(int64_t n, int64_t per_cta, int per_sm = 16) {
    const int64_t b = ceil_div(n, per_cta);
    const int64_t cap = (int64_t)sm_count() * per_sm;
    return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace tid
