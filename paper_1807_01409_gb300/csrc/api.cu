// Context, store and tuple-set management behind the C ABI (include/tid.h).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>

#include "lookback.cuh"
#include "ops.cuh"

namespace tid {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int fail_cuda(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a non-sticky error so later calls can proceed
    if (e == cudaErrorMemoryAllocation) return fail(TID_ERR_OOM, "%s: out of device memory", what);
    return fail(TID_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_err.clear(); }

// One GPU per process: launch shapes and shared-memory opt-ins are worked out
// once per process, on the device of its first context (or no-alloc scan).
static std::atomic<int> g_device{-1};

int sm_count() {
    static std::atomic<int> cached[64];  // zero: not yet queried
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    int v = dev < 64 ? cached[dev].load(std::memory_order_relaxed) : 0;
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        if (dev < 64) cached[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

int claim_device(int device) {
    int first = -1;
    if (g_device.compare_exchange_strong(first, device) || first == device) return TID_OK;
    return fail(TID_ERR_ARG, "device %d: this process already runs on device %d (one GPU per process)", device,
                first);
}

int launch_check(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, what);
    return TID_OK;
}

DeviceGuard::DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
}
DeviceGuard::~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------
int dev_alloc(tid_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    const int64_t fa = ctx->fail_after.load(std::memory_order_relaxed);
    if (fa >= 0 && ctx->allocs.fetch_add(1, std::memory_order_relaxed) >= fa)
        return fail(TID_ERR_OOM, "device allocation refused (injected failure)");
    if (bytes == 0) bytes = 256;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail_cuda(e, "device allocation");
    }
    return TID_OK;
}

void dev_free(tid_ctx *ctx, void *p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

// The context's look-back scratch, grown on demand to >= `words` status words
// (new words are zeroed, i.e. "not ready" for every epoch) plus a ticket
// counter that is 0 between launches.
int ctx_scratch(tid_ctx *ctx, size_t words, LbScratch *sc) {
    if (words > ctx->lb_cap) {
        size_t want = 1024;
        while (want < words) want *= 2;
        if (ctx->lb_status) dev_free(ctx, ctx->lb_status);
        ctx->lb_status = nullptr;
        ctx->lb_cap = 0;
        void *p = nullptr;
        TID_TRY(dev_alloc(ctx, &p, want * sizeof(unsigned long long) + 256));
        TID_TRY_CUDA(cudaMemsetAsync(p, 0, want * sizeof(unsigned long long) + 256, ctx->stream),
                     "clear look-back scratch");
        ctx->lb_status = (unsigned long long *)p;
        ctx->lb_ticket = (unsigned int *)((char *)p + want * sizeof(unsigned long long));
        ctx->lb_cap = want;
    }
    sc->status = ctx->lb_status;
    sc->cap = ctx->lb_cap;
    sc->ticket = ctx->lb_ticket;
    sc->err = ctx->err_dev;
    sc->epoch = &ctx->epoch;
    return TID_OK;
}

// Look-back state for one launch of `num_tiles` tiles: a fresh epoch, so the
// status words of earlier launches read as "not ready".
int make_lookback(const LbScratch &sc, unsigned int num_tiles, Lookback *lb) {
    if (num_tiles > sc.cap) return fail(TID_ERR_ARG, "look-back scratch holds %zu tiles, %u needed", sc.cap, num_tiles);
    unsigned e = (*sc.epoch + 1) & ((1u << 30) - 1);
    if (e == 0) e = 1;
    *sc.epoch = e;
    lb->status = sc.status;
    lb->ticket = sc.ticket;
    lb->epoch = e;
    lb->num_tiles = num_tiles;
    lb->err = sc.err;
    return TID_OK;
}

int lookback_scratch(tid_ctx *ctx, unsigned int num_tiles, Lookback *lb) {
    LbScratch sc{};
    TID_TRY(ctx_scratch(ctx, num_tiles, &sc));
    return make_lookback(sc, num_tiles, lb);
}

// ---------------------------------------------------------------------------
// row-count slots (mapped pinned host memory)
// ---------------------------------------------------------------------------
static constexpr int SLAB_SLOTS = 4096;

static void sweep_pending(tid_ctx *ctx, bool wait) {
    auto &pend = ctx->pending;
    size_t w = 0;
    for (size_t i = 0; i < pend.size(); ++i) {
        cudaError_t q = wait ? cudaEventSynchronize(pend[i].ev) : cudaEventQuery(pend[i].ev);
        if (q == cudaSuccess || q != cudaErrorNotReady) {
            cudaEventDestroy(pend[i].ev);
            ctx->free_slots.push_back({pend[i].slot.slab, pend[i].slot.index});
        } else {
            pend[w++] = pend[i];
        }
    }
    pend.resize(w);
}

static int slot_acquire(tid_ctx *ctx, Slot *s) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->free_slots.empty()) sweep_pending(ctx, false);
    if (ctx->free_slots.empty()) {
        void *h = nullptr;
        TID_TRY_CUDA(cudaHostAlloc(&h, SLAB_SLOTS * sizeof(int64_t), cudaHostAllocMapped),
                     "pinned slot slab");
        void *d = nullptr;
        cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
        if (e != cudaSuccess) {
            cudaFreeHost(h);
            return fail_cuda(e, "mapped slot slab");
        }
        const int slab = (int)ctx->slabs_host.size();
        ctx->slabs_host.push_back((int64_t *)h);
        ctx->slabs_dev.push_back((int64_t *)d);
        for (int i = SLAB_SLOTS - 1; i >= 0; --i) ctx->free_slots.push_back({slab, i});
    }
    auto si = ctx->free_slots.back();
    ctx->free_slots.pop_back();
    s->slab = si.first;
    s->index = si.second;
    s->host = ctx->slabs_host[si.first] + si.second;
    s->dev = ctx->slabs_dev[si.first] + si.second;
    *(volatile int64_t *)s->host = -1;
    return TID_OK;
}

// ---------------------------------------------------------------------------
// sets
// ---------------------------------------------------------------------------
static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int set_alloc(tid_ctx *ctx, int k, const int8_t *vars, int64_t cap, tid_set **out) {
    *out = nullptr;
    if (k < 1 || k > TID_MAX_COLS) return fail(TID_ERR_ARG, "set with %d columns", k);
    if (cap < 0) cap = 0;
    tid_set *s = new (std::nothrow) tid_set();
    if (!s) return fail(TID_ERR_OOM, "host allocation");
    s->ctx = ctx;
    s->k = k;
    for (int c = 0; c < k; ++c) s->vars[c] = vars[c];
    s->cap = cap;
    const size_t colb = align_up((size_t)cap * sizeof(int32_t), 256);
    const size_t bytes = colb * (size_t)k + 256;
    int rc = dev_alloc(ctx, &s->block, bytes);
    if (rc != TID_OK) {
        delete s;
        return rc;
    }
    for (int c = 0; c < k; ++c) s->col[c] = (int32_t *)((char *)s->block + colb * c);
    s->d_rows = (int64_t *)((char *)s->block + colb * k);
    rc = slot_acquire(ctx, &s->slot);
    if (rc == TID_OK) {
        cudaError_t e = cudaEventCreateWithFlags(&s->ready, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            s->ready = nullptr;
            rc = fail_cuda(e, "event");
        }
    }
    if (rc != TID_OK) {
        set_free(s);
        return rc;
    }
    *out = s;
    return TID_OK;
}

int set_view(tid_ctx *ctx, SharedBlock *sb, int32_t *col, int64_t *d_rows, int64_t rows, tid_set **out) {
    *out = nullptr;
    tid_set *s = new (std::nothrow) tid_set();
    if (!s) return fail(TID_ERR_OOM, "host allocation");
    s->ctx = ctx;
    s->k = 1;
    s->vars[0] = -1;
    s->cap = rows;
    s->col[0] = col;
    s->d_rows = d_rows;
    s->rows_known = rows;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        s->shared = sb;
        ++sb->refs;
    }
    *out = s;
    return TID_OK;
}

int set_ready(tid_set *set) {
    if (!set->ready) return TID_OK;  // a view: its producer is waited for through the stream
    TID_TRY_CUDA(cudaEventRecord(set->ready, set->ctx->stream), "event record");
    return TID_OK;
}

int check_ctx_error(tid_ctx *ctx) {
    int e = *(volatile int *)ctx->err_host;
    if (e != 0) {
        *(volatile int *)ctx->err_host = 0;
        // a launch that gave up may leave the ticket counter off zero
        if (ctx->lb_ticket) cudaMemsetAsync(ctx->lb_ticket, 0, sizeof(unsigned int), ctx->stream);
        if (e == TID_ERR_TIMEOUT) return fail(TID_ERR_TIMEOUT, "an in-kernel wait gave up");
        return fail(e, "kernel reported error %d", e);
    }
    return TID_OK;
}

// rows x k row-major from k columns
__global__ void k_interleave(const int32_t *const *cols, int k, const int64_t *d_rows, int32_t *out) {
    const int64_t n = *d_rows;
    const int64_t total = n * k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / k;
        const int c = (int)(i - r * k);
        out[i] = cols[c][r];
    }
}

}  // namespace tid


// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace tid;

extern "C" const char *tid_last_error(void) { return g_err.c_str(); }

extern "C" int tid_ctx_create(int device, void *cuda_stream, tid_ctx **out) {
    clear_error();
    if (!out) return fail(TID_ERR_ARG, "tid_ctx_create: null out");
    *out = nullptr;
    int ndev = 0;
    TID_TRY_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(TID_ERR_ARG, "tid_ctx_create: no device %d", device);
    TID_TRY(claim_device(device));
    DeviceGuard g(device);
    tid_ctx *c = new (std::nothrow) tid_ctx();
    if (!c) return fail(TID_ERR_OOM, "host allocation");
    c->device = device;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = true;
    }
    if (e == cudaSuccess) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&c->pool, &props);
        if (e == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    void *h = nullptr;
    if (e == cudaSuccess) e = cudaHostAlloc(&h, 256, cudaHostAllocMapped);
    if (e == cudaSuccess) {
        c->err_host = (int *)h;
        *c->err_host = 0;
        void *d = nullptr;
        e = cudaHostGetDevicePointer(&d, h, 0);
        c->err_dev = (int *)d;
    }
    if (e != cudaSuccess) {
        int rc = fail_cuda(e, "tid_ctx_create");
        if (c->err_host) cudaFreeHost(c->err_host);
        if (c->pool) cudaMemPoolDestroy(c->pool);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
        delete c;
        return rc;
    }
    *out = c;
    return TID_OK;
}

extern "C" int tid_ctx_sync(tid_ctx *ctx) {
    clear_error();
    tid::Range nvtx_range("tid_ctx_sync");
    if (!ctx) return fail(TID_ERR_ARG, "tid_ctx_sync: null ctx");
    DeviceGuard g(ctx->device);
    TID_TRY_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    return check_ctx_error(ctx);
}

extern "C" int tid_ctx_destroy(tid_ctx *ctx) {
    clear_error();
    if (!ctx) return TID_OK;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        sweep_pending(ctx, true);
    }
    if (ctx->lb_status) cudaFreeAsync(ctx->lb_status, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    for (auto *h : ctx->slabs_host) cudaFreeHost(h);
    if (ctx->err_host) cudaFreeHost(ctx->err_host);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return TID_OK;
}

namespace {
// One CTA arrives at a barrier of two that no other CTA reaches: the library's
// bounded wait gives up after `limit` polls and sets TID_ERR_TIMEOUT.
__global__ void k_wait_for_nothing(unsigned *counter, int *err, unsigned limit) {
    tid::grid_barrier(counter, 2u, err, limit);
}
}  // namespace

extern "C" int tid_ctx_test_bounded_wait(tid_ctx *ctx, int64_t polls) {
    clear_error();
    if (!ctx) return fail(TID_ERR_ARG, "tid_ctx_test_bounded_wait: null context");
    if (polls < 1 || polls > (int64_t)LB_SPIN_LIMIT)
        return fail(TID_ERR_ARG, "tid_ctx_test_bounded_wait: polls = %lld", (long long)polls);
    DeviceGuard g(ctx->device);
    void *counter = nullptr;
    TID_TRY(dev_alloc(ctx, &counter, 256));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx->stream);
    if (e == cudaSuccess) {
        k_wait_for_nothing<<<1, 32, 0, ctx->stream>>>((unsigned *)counter, ctx->err_dev, (unsigned)polls);
        e = cudaGetLastError();
    }
    dev_free(ctx, counter);
    if (e != cudaSuccess) return fail_cuda(e, "tid_ctx_test_bounded_wait");
    return tid_ctx_sync(ctx);
}

extern "C" int tid_ctx_inject_alloc_failure(tid_ctx *ctx, int64_t after) {
    clear_error();
    if (!ctx) return fail(TID_ERR_ARG, "tid_ctx_inject_alloc_failure: null context");
    ctx->allocs.store(0);
    ctx->fail_after.store(after < 0 ? -1 : after);
    return TID_OK;
}

namespace {
// *unsorted = 1 if some triple is smaller, in (s, p, o) order, than the one
// before it
__global__ void k_spo_unsorted(const int32_t *__restrict__ s, const int32_t *__restrict__ p,
                               const int32_t *__restrict__ o, int64_t n, int32_t *__restrict__ unsorted) {
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s0 = s[i - 1], s1 = s[i];
        if (s0 != s1) {
            bad = bad || s0 > s1;
            continue;
        }
        const int32_t p0 = p[i - 1], p1 = p[i];
        bad = bad || p0 > p1 || (p0 == p1 && o[i - 1] > o[i]);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *unsorted = 1;
}
}  // namespace

namespace tid {
bool store_spo_sorted(const tid_store *st) {
    if (st->spo_sorted < 0) {
        int32_t h = 1;
        DeviceGuard g(st->ctx->device);
        cudaError_t e = cudaMemcpyAsync(&h, st->d_unsorted, sizeof h, cudaMemcpyDeviceToHost, st->ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st->ctx->stream);
        if (e != cudaSuccess) return false;  // unknown: take the general path
        st->spo_sorted = h == 0 ? 1 : 0;
    }
    return st->spo_sorted == 1;
}
}  // namespace tid

extern "C" int tid_load(tid_ctx *ctx, const int32_t *s, const int32_t *p, const int32_t *o,
                        int64_t n, int where, int copy, tid_store **out) {
    clear_error();
    tid::Range nvtx_range("tid_load");
    if (!ctx || !out) return fail(TID_ERR_ARG, "tid_load: null argument");
    *out = nullptr;
    if (n < 0 || n > INT32_MAX) return fail(TID_ERR_ARG, "tid_load: n = %lld out of range", (long long)n);
    if (n > 0 && (!s || !p || !o)) return fail(TID_ERR_ARG, "tid_load: null column");
    if (where != TID_HOST && where != TID_DEVICE) return fail(TID_ERR_ARG, "tid_load: bad `where`");
    DeviceGuard g(ctx->device);
    tid_store *st = new (std::nothrow) tid_store();
    if (!st) return fail(TID_ERR_OOM, "host allocation");
    st->ctx = ctx;
    st->n = n;
    if (where == TID_DEVICE && !copy) {
        st->s = s;
        st->p = p;
        st->o = o;
    } else {
        const size_t colb = align_up((size_t)n * sizeof(int32_t), 256);
        int rc = dev_alloc(ctx, &st->owned, 3 * colb);
        if (rc != TID_OK) {
            delete st;
            return rc;
        }
        int32_t *base = (int32_t *)st->owned;
        int32_t *cs = base, *cp = (int32_t *)((char *)base + colb), *co = (int32_t *)((char *)base + 2 * colb);
        const cudaMemcpyKind kind = where == TID_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        cudaError_t e = cudaSuccess;
        if (n > 0) {
            e = cudaMemcpyAsync(cs, s, (size_t)n * 4, kind, ctx->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(cp, p, (size_t)n * 4, kind, ctx->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(co, o, (size_t)n * 4, kind, ctx->stream);
        }
        if (e != cudaSuccess) {
            dev_free(ctx, st->owned);
            delete st;
            return fail_cuda(e, "tid_load copy");
        }
        st->s = cs;
        st->p = cp;
        st->o = co;
    }
    st->aligned16 = ((uintptr_t)st->s % 16 == 0) && ((uintptr_t)st->p % 16 == 0) &&
                    ((uintptr_t)st->o % 16 == 0);
    // the order check: one read of the store, queued like the copies
    int rc = dev_alloc(ctx, (void **)&st->d_unsorted, sizeof(int32_t));
    if (rc == TID_OK) {
        cudaError_t e = cudaMemsetAsync(st->d_unsorted, 0, sizeof(int32_t), ctx->stream);
        if (e != cudaSuccess) rc = fail_cuda(e, "tid_load");
    }
    if (rc == TID_OK && n > 1) {
        k_spo_unsorted<<<grid_for(n, 256, 8), 256, 0, ctx->stream>>>(st->s, st->p, st->o, n, st->d_unsorted);
        rc = launch_check("k_spo_unsorted");
    }
    if (rc != TID_OK) {
        if (st->d_unsorted) dev_free(ctx, st->d_unsorted);
        if (st->owned) dev_free(ctx, st->owned);
        delete st;
        return rc;
    }
    *out = st;
    return TID_OK;
}

extern "C" int tid_store_info(const tid_store *st, int64_t *n, const int32_t **s, const int32_t **p,
                              const int32_t **o) {
    clear_error();
    if (!st) return fail(TID_ERR_ARG, "tid_store_info: null store");
    if (n) *n = st->n;
    if (s) *s = st->s;
    if (p) *p = st->p;
    if (o) *o = st->o;
    return TID_OK;
}

extern "C" int tid_store_free(tid_store *st) {
    clear_error();
    if (!st) return TID_OK;
    DeviceGuard g(st->ctx->device);
    if (st->d_unsorted) dev_free(st->ctx, st->d_unsorted);
    if (st->owned) dev_free(st->ctx, st->owned);
    delete st;
    return TID_OK;
}

namespace tid {
int set_rows_host(tid_set *set, int64_t *rows) {
    if (set->rows_known < 0) {
        DeviceGuard g(set->ctx->device);
        TID_TRY_CUDA(cudaEventSynchronize(set->ready), "wait for set");
        TID_TRY(check_ctx_error(set->ctx));
        const int64_t r = *(volatile int64_t *)set->slot.host;
        if (r < 0) return fail(TID_ERR_CUDA, "row count was not produced");
        set->rows_known = r;
    }
    *rows = set->rows_known;
    return TID_OK;
}
int set_rows_host(const tid_set *set, int64_t *rows) { return set_rows_host(const_cast<tid_set *>(set), rows); }
}  // namespace tid

extern "C" int tid_set_rows(tid_set *set, int64_t *rows) {
    clear_error();
    tid::Range nvtx_range("tid_set_rows");
    if (!set || !rows) return fail(TID_ERR_ARG, "tid_set_rows: null argument");
    return set_rows_host(set, rows);
}

extern "C" int tid_set_info(const tid_set *set, int *cols, int64_t *capacity, const int8_t **var_ids,
                            int32_t *const **dev_cols, const int64_t **dev_rows) {
    clear_error();
    if (!set) return fail(TID_ERR_ARG, "tid_set_info: null set");
    if (cols) *cols = set->k;
    if (capacity) *capacity = set->cap;
    if (var_ids) *var_ids = set->vars;
    if (dev_cols) *dev_cols = set->col;
    if (dev_rows) *dev_rows = set->d_rows;
    return TID_OK;
}

extern "C" int tid_set_to_host(tid_set *set, int32_t *buf, int64_t cap_rows, int64_t *rows_out) {
    clear_error();
    tid::Range nvtx_range("tid_set_to_host");
    if (!set) return fail(TID_ERR_ARG, "tid_set_to_host: null set");
    int64_t rows = 0;
    TID_TRY(tid_set_rows(set, &rows));
    if (rows_out) *rows_out = rows;
    if (rows > cap_rows) return fail(TID_ERR_CAPACITY, "tid_set_to_host: %lld rows > %lld", (long long)rows, (long long)cap_rows);
    if (rows == 0) return TID_OK;
    if (!buf) return fail(TID_ERR_ARG, "tid_set_to_host: null buffer");
    tid_ctx *ctx = set->ctx;
    DeviceGuard g(ctx->device);
    const size_t bytes = (size_t)rows * set->k * sizeof(int32_t);
    if (set->k == 1) {
        TID_TRY_CUDA(cudaMemcpyAsync(buf, set->col[0], bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy set");
    } else {
        void *tmp = nullptr;
        TID_TRY(dev_alloc(ctx, &tmp, align_up(bytes, 256) + sizeof(int32_t *) * TID_MAX_COLS));
        int32_t **dcols = (int32_t **)((char *)tmp + align_up(bytes, 256));
        cudaError_t e = cudaMemcpyAsync(dcols, set->col, sizeof(int32_t *) * set->k, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) {
            const int64_t blocks = ceil_div(rows * set->k, 256);
            k_interleave<<<grid_for(blocks, 1), 256, 0, ctx->stream>>>(
                dcols, set->k, set->d_rows, (int32_t *)tmp);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(buf, tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream);
        dev_free(ctx, tmp);
        if (e != cudaSuccess) return fail_cuda(e, "copy set");
    }
    TID_TRY_CUDA(cudaStreamSynchronize(ctx->stream), "copy set");
    return check_ctx_error(ctx);
}

namespace tid {
// frees a set without touching the error message (used on error paths too)
void set_free(tid_set *set) {
    if (!set) return;
    tid_ctx *ctx = set->ctx;
    DeviceGuard g(ctx->device);
    if (set->block) dev_free(ctx, set->block);
    if (set->shared) {
        SharedBlock *sb = set->shared;
        bool last;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            last = --sb->refs == 0;
        }
        if (last) {
            for (void *p : sb->ptr)
                if (p) dev_free(ctx, p);
            delete sb;
        }
    }
    if (set->slot.slab >= 0) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (set->ready) {
            // the producer may still be writing the slot: recycle it once done
            ctx->pending.push_back({set->slot, set->ready});
            set->ready = nullptr;
        } else {
            ctx->free_slots.push_back({set->slot.slab, set->slot.index});
        }
    }
    if (set->ready) cudaEventDestroy(set->ready);
    delete set;
}
}  // namespace tid

extern "C" int tid_set_free(tid_set *set) {
    clear_error();
    tid::set_free(set);
    return TID_OK;
}
