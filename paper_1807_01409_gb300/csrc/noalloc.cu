// tid_match_noalloc: the single-pattern scan for callers that may not allocate
// device memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates device
// memory) at the moment they want to run a scan: a serving process that has
// handed all free device memory to its own pool at start-up, or a latency-
// critical loop where an allocation's implicit synchronisation and
// unpredictable cost are not allowed.  They pass every input and output
// buffer themselves; the only other memory the scan needs -- the look-back
// status words, the ticket counter and an error word -- lives in one
// file-scope __device__ array of fixed size instead of a context's pool.
//
// That array exists once per GPU that loads this library and lives until the
// process exits.  Every call on a GPU shares it and it keeps the previous
// call's contents, so each call first clears all of it (one stream-ordered
// memset of 32 KB, no allocation): status words, ticket counter and error
// word start at zero whatever ran before.  After the scan a one-thread kernel
// sets *count to -1 if any wait gave up, since the caller cannot read the
// array's error word.  Two calls whose GPU work overlaps (different streams
// without an ordering between them) race on the array and give wrong results:
// order them.

#include <mutex>

#include "tid_internal.cuh"

namespace {

constexpr size_t NOALLOC_STATUS_WORDS = TID_NOALLOC_MAX_CHUNKS;
constexpr int NOALLOC_MAX_DEVICES = 64;

// [0, W): status words; word W: ticket counter (low 32 bits); word W+1: error word.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_STATUS_WORDS + 32];

struct DeviceScratch {
    bool ready = false;
    unsigned long long *base = nullptr;  // device address of g_noalloc_scratch on this GPU
    unsigned int epoch = 0;              // launch epochs used on this GPU
};

std::mutex g_mu;
DeviceScratch g_dev[NOALLOC_MAX_DEVICES];

// Once per device, with that device current: the device address of the array.
// (In host code the array's name is only a host-side stand-in.)
int device_scratch(int device, DeviceScratch **out) {
    DeviceScratch &d = g_dev[device];
    if (!d.ready) {
        tid::DeviceGuard g(device);
        unsigned long long *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return tid::fail_cuda(e, "tid_match_noalloc: scratch address");
        d.base = p;
        d.ready = true;
    }
    *out = &d;
    return TID_OK;
}

// After the scan: a wait that gave up left its code in the error word; the
// count is then -1, whatever a later tile wrote.
__global__ void k_noalloc_finish(const unsigned long long *ctl, int64_t *count) {
    if (*(const int *)(ctl + 1) != 0) *count = -1;
}

}  // namespace

extern "C" int tid_match_noalloc(int device, void *cuda_stream, const int32_t *s, const int32_t *p,
                                 const int32_t *o, int64_t n, tid_pattern pat, int32_t *out, int64_t cap,
                                 int64_t *count) {
    using namespace tid;
    clear_error();
    Range nvtx_range("tid_match_noalloc");
    if (n < 0 || n > INT32_MAX) return fail(TID_ERR_ARG, "tid_match_noalloc: n = %lld out of range", (long long)n);
    if (n > 0 && (!s || !p || !o)) return fail(TID_ERR_ARG, "tid_match_noalloc: null column");
    if (!count) return fail(TID_ERR_ARG, "tid_match_noalloc: null count");
    if (cap < 0 || (cap > 0 && !out)) return fail(TID_ERR_ARG, "tid_match_noalloc: bad output buffer");
    if (pat.s < 0 || pat.p < 0 || pat.o < 0) return fail(TID_ERR_ID, "tid_match_noalloc: negative ID in pattern");
    int ndev = 0;
    TID_TRY_CUDA(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount");
    if (device < 0 || device >= ndev || device >= NOALLOC_MAX_DEVICES)
        return fail(TID_ERR_ARG, "tid_match_noalloc: no device %d", device);
    TID_TRY(claim_device(device));

    std::lock_guard<std::mutex> lk(g_mu);
    DeviceScratch *d = nullptr;
    TID_TRY(device_scratch(device, &d));
    DeviceGuard g(device);
    const unsigned need = match_scratch_words();
    if (need > NOALLOC_STATUS_WORDS)
        return fail(TID_ERR_CAPACITY,
                    "tid_match_noalloc: this GPU runs %u scan chunks per launch, the built-in scratch holds %zu",
                    need, NOALLOC_STATUS_WORDS);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned long long *ctl = d->base + NOALLOC_STATUS_WORDS;  // ticket, error word
    TID_TRY_CUDA(cudaMemsetAsync(d->base, 0, sizeof(g_noalloc_scratch), st), "tid_match_noalloc: clear scratch");
    TID_TRY_CUDA(cudaMemsetAsync(count, 0xFF, sizeof(int64_t), st), "tid_match_noalloc: clear count");
    LbScratch sc{};
    sc.status = d->base;
    sc.cap = NOALLOC_STATUS_WORDS;
    sc.ticket = (unsigned int *)ctl;
    sc.err = (int *)(ctl + 1);
    sc.epoch = &d->epoch;
    const bool aligned16 = ((uintptr_t)s % 16 == 0) && ((uintptr_t)p % 16 == 0) && ((uintptr_t)o % 16 == 0);
    TID_TRY(launch_match(st, s, p, o, n, aligned16, pat.s, pat.p, pat.o, out, cap, count, count, sc));
    k_noalloc_finish<<<1, 1, 0, st>>>(ctl, count);
    return launch_check("k_noalloc_finish");
}
