// tid_server: a request loop over a resident store with continuous batching
// (behaviour specified with the declarations in tid.h).
//
// Host-side structure:
//  * one FIFO queue of requests under one mutex; workers admit from its head
//    (estimated bytes against the budget, at most max_wave per wave);
//  * each worker owns a context (stream + memory pool) and a borrowed view of
//    the store, so waves of different workers overlap on the device;
//  * a wave: (batch_scans) every MATCH node of the wave -> one tid_match_batch;
//    then the index requests' lists go to host, smallest first, in chunks
//    through two fixed pinned buffers (the copy of one chunk overlaps the host
//    copy of the previous one) and each request finishes as soon as its rows
//    are on the host; then each plan runs the rest of its nodes (exec_plan)
//    and is copied to host;
//  * estimates come from sorted value samples of the three columns.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ops.cuh"

namespace {

using namespace tid;

constexpr int MAX_WORKERS = 16;
constexpr size_t STAGE_ROWS = (size_t)1 << 24;  // rows per pinned staging buffer (64 MB)
constexpr int64_t SAMPLE_MAX = 1 << 20;

struct Request {
    int64_t id = 0;
    int kind = 0;
    std::vector<tid_plan_node> nodes;
    int64_t arrival_ns = 0;
    int64_t est_bytes = 0;
    bool waited = false;  // held at the queue's head by the budget
    // result
    bool done = false;
    int status = TID_OK;
    int cols = 0;
    int8_t vars[TID_MAX_COLS] = {0};
    int64_t rows = 0;
    std::unique_ptr<int32_t[]> data;  // rows x cols, row-major (not zero-filled before it is written)
    int64_t latency_ns = 0;
};

struct Worker {
    tid_ctx *ctx = nullptr;
    tid_store *st = nullptr;
    std::thread th;
    int32_t *staging[2] = {nullptr, nullptr};  // pinned host buffers for index results, STAGE_ROWS each
    cudaEvent_t copied[2] = {nullptr, nullptr};
};

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

struct tid_server {
    int device = 0;
    tid_server_config cfg{};
    const int32_t *s = nullptr, *p = nullptr, *o = nullptr;
    int64_t n = 0;
    // estimator: sorted sampled values of each column and the scale sample -> store
    std::vector<int32_t> sample[3];
    double scale = 1.0;

    std::mutex mu;
    std::condition_variable cv_work;  // queue changed, memory freed, or stop
    std::condition_variable cv_done;  // a request finished
    std::deque<Request *> queue;
    // shared: a waiter keeps its request alive if another thread releases it
    std::unordered_map<int64_t, std::shared_ptr<Request>> reqs;
    int64_t next_id = 1;
    int64_t admitted_bytes = 0;
    int admitted_reqs = 0;
    bool stop = false;
    tid_server_stats stats{};
    Worker workers[MAX_WORKERS];
};

namespace {

double est_pattern_rows(const tid_server *S, const tid_pattern &pat) {
    const int32_t key[3] = {pat.s, pat.p, pat.o};
    double best = (double)S->n;
    for (int c = 0; c < 3; ++c) {
        if (key[c] == 0) continue;
        const auto &v = S->sample[c];
        const auto r = std::equal_range(v.begin(), v.end(), key[c]);
        const double cnt = (double)(r.second - r.first);
        best = std::min(best, std::max(cnt, 0.5) * S->scale);  // unseen: half a sample step
    }
    return std::max(1.0, best);
}

int64_t est_request_bytes(const tid_server *S, int kind, const std::vector<tid_plan_node> &nodes) {
    if (kind == TID_REQ_INDEX) return (int64_t)(4.0 * est_pattern_rows(S, nodes[0].pattern));
    const int n = (int)nodes.size();
    std::vector<double> rows(n, 0.0);
    std::vector<int> cols(n, 1);
    double bytes = 0.0;
    for (int i = 0; i < n; ++i) {
        const tid_plan_node &nd = nodes[i];
        switch (nd.op) {
            case TID_OP_MATCH: {
                rows[i] = est_pattern_rows(S, nd.pattern);
                int k = 0;
                for (int j = 0; j < 3; ++j) k += nd.pattern.var[j] >= 0;
                cols[i] = std::max(1, k);
                bytes += rows[i] * 4.0;  // the index list
                break;
            }
            case TID_OP_FILTER:
            case TID_OP_PROJECT:
                rows[i] = rows[nd.in[0]];
                cols[i] = nd.op == TID_OP_PROJECT ? std::max(1, (int)nd.n_vars) : cols[nd.in[0]];
                break;
            case TID_OP_JOIN:
                rows[i] = std::max(rows[nd.in[0]], rows[nd.in[1]]);
                cols[i] = std::min(TID_MAX_COLS, cols[nd.in[0]] + cols[nd.in[1]]);
                break;
            case TID_OP_UNION:
                for (int j = 0; j < nd.n_in; ++j) {
                    rows[i] += rows[nd.in[j]];
                    cols[i] = std::max(cols[i], cols[nd.in[j]]);
                }
                break;
        }
        bytes += rows[i] * 4.0 * (cols[i] + 1);
    }
    return (int64_t)std::min(bytes, 4.0e13);
}

// Requests at the queue's head that fit (called with the lock held).
void admit(tid_server *S, std::vector<Request *> &wave) {
    while (!S->queue.empty() && (int)wave.size() < S->cfg.max_wave) {
        Request *r = S->queue.front();
        const bool alone = S->admitted_reqs == 0 && wave.empty();
        if (S->cfg.budget_bytes > 0 && !alone && S->admitted_bytes + r->est_bytes > S->cfg.budget_bytes) {
            if (!r->waited) S->stats.budget_waits++;
            r->waited = true;
            break;
        }
        S->queue.pop_front();
        S->admitted_bytes += r->est_bytes;
        S->admitted_reqs++;
        wave.push_back(r);
    }
    if (!wave.empty()) {
        S->stats.waves++;
        S->stats.max_wave_seen = std::max<int64_t>(S->stats.max_wave_seen, (int64_t)wave.size());
        S->stats.peak_admitted_bytes = std::max(S->stats.peak_admitted_bytes, S->admitted_bytes);
    }
}

void finish(tid_server *S, Request *r) {
    std::lock_guard<std::mutex> lk(S->mu);
    r->latency_ns = now_ns() - r->arrival_ns;
    r->done = true;
    S->admitted_bytes -= r->est_bytes;
    S->admitted_reqs--;
    if (r->status == TID_OK) S->stats.completed++;
    else S->stats.failed++;
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

int set_to_request(tid_set *set, Request *r) {
    int64_t rows = 0;
    TID_TRY(set_rows_host(set, &rows));
    r->cols = set->k;
    for (int c = 0; c < set->k; ++c) r->vars[c] = set->vars[c];
    r->rows = rows;
    r->data.reset(new (std::nothrow) int32_t[std::max<size_t>(1, (size_t)rows * set->k)]);
    if (!r->data) return fail(TID_ERR_OOM, "host allocation of a result");
    if (rows == 0) return TID_OK;
    int64_t got = 0;
    return tid_set_to_host(set, r->data.get(), rows, &got);
}

// An index list (n rows on the device) into dst on the host, in chunks through
// the worker's two pinned buffers: the copy into one buffer runs while the
// previous chunk is copied out of the other.
int list_to_host(Worker &W, cudaStream_t st, const int32_t *src, size_t n, int32_t *dst) {
    size_t prev_off = 0, prev_len = 0;
    int prev_buf = -1;
    for (size_t off = 0, k = 0; off < n; off += STAGE_ROWS, ++k) {
        const int b = (int)(k & 1);
        const size_t len = std::min(STAGE_ROWS, n - off);
        TID_TRY_CUDA(cudaMemcpyAsync(W.staging[b], src + off, len * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
                     "index result copy");
        TID_TRY_CUDA(cudaEventRecord(W.copied[b], st), "index result copy");
        if (prev_buf >= 0) {
            TID_TRY_CUDA(cudaEventSynchronize(W.copied[prev_buf]), "index result copy");
            std::memcpy(dst + prev_off, W.staging[prev_buf], prev_len * sizeof(int32_t));
        }
        prev_buf = b;
        prev_off = off;
        prev_len = len;
    }
    if (prev_buf >= 0) {
        TID_TRY_CUDA(cudaEventSynchronize(W.copied[prev_buf]), "index result copy");
        std::memcpy(dst + prev_off, W.staging[prev_buf], prev_len * sizeof(int32_t));
    }
    return TID_OK;
}

void run_wave(tid_server *S, Worker &W, std::vector<Request *> &wave) {
    Range nvtx_range("tid_server_wave");
    tid_ctx *ctx = W.ctx;
    const tid_store *st = W.st;
    const int nw = (int)wave.size();
    std::vector<std::vector<tid_set *>> matched(nw);
    for (int i = 0; i < nw; ++i) matched[i].assign(wave[i]->nodes.size(), nullptr);

    // 1) the wave's searches
    if (S->cfg.batch_scans) {
        std::vector<tid_pattern> pats;
        std::vector<std::pair<int, int>> where;
        for (int i = 0; i < nw; ++i)
            for (size_t j = 0; j < wave[i]->nodes.size(); ++j)
                if (wave[i]->nodes[j].op == TID_OP_MATCH) {
                    pats.push_back(wave[i]->nodes[j].pattern);
                    where.push_back({i, (int)j});
                }
        std::vector<tid_set *> outs(pats.size(), nullptr);
        const int rc = pats.empty() ? TID_OK : tid_match_batch(ctx, st, pats.data(), (int)pats.size(), outs.data());
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.scan_patterns += (int64_t)pats.size();
        }
        if (rc != TID_OK) {
            for (Request *r : wave) {
                r->status = rc;
                finish(S, r);
            }
            return;
        }
        for (size_t q = 0; q < pats.size(); ++q) matched[where[q].first][where[q].second] = outs[q];
    } else {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request *r : wave)
            for (auto &nd : r->nodes) S->stats.scan_patterns += nd.op == TID_OP_MATCH;
    }

    // 2) index requests: their lists to host, smallest first, each request
    //    finished as soon as its rows are there
    std::vector<int> idx_reqs;
    std::vector<tid_set *> idx_sets;
    for (int i = 0; i < nw; ++i) {
        Request *r = wave[i];
        if (r->kind != TID_REQ_INDEX) continue;
        tid_set *set = matched[i][0];
        matched[i][0] = nullptr;
        int rc = set ? TID_OK : tid_match(ctx, st, r->nodes[0].pattern, &set);
        int64_t rows = 0;
        if (rc == TID_OK) rc = set_rows_host(set, &rows);
        if (rc != TID_OK) {
            if (set) set_free(set);
            r->status = rc;
            finish(S, r);
            continue;
        }
        r->cols = 1;
        r->vars[0] = -1;
        r->rows = rows;
        idx_reqs.push_back(i);
        idx_sets.push_back(set);
    }
    std::vector<size_t> order(idx_reqs.size());
    for (size_t q = 0; q < order.size(); ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t b) { return wave[idx_reqs[a]]->rows < wave[idx_reqs[b]]->rows; });
    int copy_rc = check_ctx_error(ctx);
    for (size_t q : order) {
        Request *r = wave[idx_reqs[q]];
        int rc = copy_rc;
        if (rc == TID_OK) {
            r->data.reset(new (std::nothrow) int32_t[std::max<int64_t>(1, r->rows)]);
            rc = r->data ? TID_OK : fail(TID_ERR_OOM, "host allocation of a result");
        }
        if (rc == TID_OK) rc = list_to_host(W, ctx->stream, idx_sets[q]->col[0], (size_t)r->rows, r->data.get());
        if (rc != TID_OK) copy_rc = rc;
        set_free(idx_sets[q]);
        r->status = rc;
        finish(S, r);
    }

    // 3) plans: the rest of each plan, then its result to host
    for (int i = 0; i < nw; ++i) {
        Request *r = wave[i];
        if (r->kind != TID_REQ_PLAN) continue;
        tid_set *out = nullptr;
        int rc = exec_plan(ctx, st, r->nodes.data(), (int)r->nodes.size(), matched[i].data(), &out);
        if (rc == TID_OK) rc = set_to_request(out, r);
        if (out) set_free(out);
        r->status = rc;
        finish(S, r);
    }
    for (auto &m : matched)
        for (tid_set *x : m)
            if (x) set_free(x);
}

void worker_loop(tid_server *S, int w) {
    Worker &W = S->workers[w];
    DeviceGuard g(S->device);
    for (;;) {
        std::vector<Request *> wave;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (;;) {
                admit(S, wave);
                if (!wave.empty()) break;
                if (S->stop && S->queue.empty()) return;
                S->cv_work.wait(lk);
            }
        }
        run_wave(S, W, wave);
    }
}

int make_sample(tid_server *S) {
    const int64_t n = S->n;
    const int64_t m = std::min<int64_t>(n, SAMPLE_MAX);
    if (m == 0) return TID_OK;
    const int64_t stride = n / m;
    S->scale = (double)n / (double)m;
    const int32_t *cols[3] = {S->s, S->p, S->o};
    for (int c = 0; c < 3; ++c) {
        S->sample[c].resize(m);
        // every stride-th value: one strided copy per column
        TID_TRY_CUDA(cudaMemcpy2D(S->sample[c].data(), sizeof(int32_t), cols[c], (size_t)stride * sizeof(int32_t),
                                  sizeof(int32_t), (size_t)m, cudaMemcpyDeviceToHost),
                     "store sample");
        std::sort(S->sample[c].begin(), S->sample[c].end());
    }
    return TID_OK;
}

void destroy_workers(tid_server *S) {
    for (auto &W : S->workers) {
        if (W.st) tid_store_free(W.st);
        if (W.ctx) tid_ctx_destroy(W.ctx);
        for (int b = 0; b < 2; ++b) {
            if (W.staging[b]) cudaFreeHost(W.staging[b]);
            if (W.copied[b]) cudaEventDestroy(W.copied[b]);
        }
        W = Worker();
    }
}

}  // namespace

extern "C" int64_t tid_server_now_ns(void) { return now_ns(); }

extern "C" int tid_server_create(int device, const int32_t *s, const int32_t *p, const int32_t *o, int64_t n,
                                 const tid_server_config *cfg, tid_server **out) {
    clear_error();
    if (!out || !cfg) return fail(TID_ERR_ARG, "tid_server_create: null argument");
    *out = nullptr;
    if (n < 0 || n > INT32_MAX) return fail(TID_ERR_ARG, "tid_server_create: n = %lld", (long long)n);
    if (n > 0 && (!s || !p || !o)) return fail(TID_ERR_ARG, "tid_server_create: null column");
    if (cfg->workers < 1 || cfg->workers > MAX_WORKERS || cfg->max_wave < 1 || cfg->budget_bytes < 0 ||
        (cfg->batch_scans != 0 && cfg->batch_scans != 1))
        return fail(TID_ERR_ARG, "tid_server_create: bad configuration");
    std::unique_ptr<tid_server> S(new (std::nothrow) tid_server());
    if (!S) return fail(TID_ERR_OOM, "host allocation");
    S->device = device;
    S->cfg = *cfg;
    S->s = s;
    S->p = p;
    S->o = o;
    S->n = n;
    for (int w = 0; w < cfg->workers; ++w) {
        Worker &W = S->workers[w];
        int rc = tid_ctx_create(device, nullptr, &W.ctx);
        if (rc == TID_OK) rc = tid_load(W.ctx, s, p, o, n, TID_DEVICE, 0, &W.st);
        for (int b = 0; b < 2 && rc == TID_OK; ++b) {
            DeviceGuard g(device);
            void *h = nullptr;
            cudaError_t e = cudaHostAlloc(&h, STAGE_ROWS * sizeof(int32_t), cudaHostAllocDefault);
            if (e == cudaSuccess) {
                W.staging[b] = (int32_t *)h;
                e = cudaEventCreateWithFlags(&W.copied[b], cudaEventDisableTiming);
            }
            if (e != cudaSuccess) rc = fail_cuda(e, "tid_server_create: staging buffers");
        }
        if (rc != TID_OK) {
            destroy_workers(S.get());
            return rc;
        }
    }
    {
        DeviceGuard g(device);
        // the columns may still be being written on another stream: wait for the
        // device once, before the sample and before any worker reads them
        const cudaError_t e = cudaDeviceSynchronize();
        const int rc = e != cudaSuccess ? fail_cuda(e, "tid_server_create: device synchronize") : make_sample(S.get());
        if (rc != TID_OK) {
            destroy_workers(S.get());
            return rc;
        }
    }
    for (int w = 0; w < cfg->workers; ++w) S->workers[w].th = std::thread(worker_loop, S.get(), w);
    *out = S.release();
    return TID_OK;
}

extern "C" int tid_server_submit(tid_server *S, int kind, const tid_plan_node *nodes, int n_nodes, int64_t arrival_ns,
                                 int64_t *id) {
    clear_error();
    if (!S || !nodes || !id) return fail(TID_ERR_ARG, "tid_server_submit: null argument");
    if (kind == TID_REQ_INDEX) {
        if (n_nodes != 1 || nodes[0].op != TID_OP_MATCH)
            return fail(TID_ERR_ARG, "tid_server_submit: an index request is one MATCH node");
        const tid_pattern &pt = nodes[0].pattern;
        if (pt.s < 0 || pt.p < 0 || pt.o < 0) return fail(TID_ERR_ID, "tid_server_submit: negative ID in pattern");
    } else if (kind == TID_REQ_PLAN) {
        TID_TRY(validate_plan(nodes, n_nodes));
    } else {
        return fail(TID_ERR_ARG, "tid_server_submit: unknown kind %d", kind);
    }
    std::shared_ptr<Request> r;
    try {
        r = std::make_shared<Request>();
    } catch (const std::bad_alloc &) {
        return fail(TID_ERR_OOM, "host allocation");
    }
    r->kind = kind;
    r->nodes.assign(nodes, nodes + n_nodes);
    r->arrival_ns = arrival_ns > 0 ? arrival_ns : now_ns();
    r->est_bytes = est_request_bytes(S, kind, r->nodes);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return fail(TID_ERR_ARG, "tid_server_submit: server is stopping");
        r->id = S->next_id++;
        *id = r->id;
        S->queue.push_back(r.get());
        S->reqs[r->id] = std::move(r);
        S->stats.submitted++;
    }
    S->cv_work.notify_one();
    return TID_OK;
}

extern "C" int tid_server_wait(tid_server *S, int64_t id, int64_t timeout_ms) {
    clear_error();
    Range nvtx_range("tid_server_wait");
    if (!S) return fail(TID_ERR_ARG, "tid_server_wait: null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return fail(TID_ERR_ARG, "tid_server_wait: unknown request %lld", (long long)id);
    const std::shared_ptr<Request> keep = it->second;  // alive across the wait
    Request *r = keep.get();
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, [&] { return r->done; });
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; })) {
        return fail(TID_ERR_TIMEOUT, "tid_server_wait: request %lld not finished", (long long)id);
    }
    return TID_OK;
}

extern "C" int tid_server_result(tid_server *S, int64_t id, int *status, int *cols, int8_t *vars, int64_t *rows,
                                 const int32_t **data, int64_t *latency_ns) {
    clear_error();
    if (!S) return fail(TID_ERR_ARG, "tid_server_result: null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || !it->second->done)
        return fail(TID_ERR_ARG, "tid_server_result: request %lld unknown or unfinished", (long long)id);
    const Request *r = it->second.get();
    if (status) *status = r->status;
    if (cols) *cols = r->cols;
    if (vars)
        for (int c = 0; c < r->cols; ++c) vars[c] = r->vars[c];
    if (rows) *rows = r->rows;
    if (data) *data = r->data.get();
    if (latency_ns) *latency_ns = r->latency_ns;
    return TID_OK;
}

extern "C" int tid_server_release(tid_server *S, int64_t id) {
    clear_error();
    if (!S) return fail(TID_ERR_ARG, "tid_server_release: null server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || !it->second->done)
        return fail(TID_ERR_ARG, "tid_server_release: request %lld unknown or unfinished", (long long)id);
    S->reqs.erase(it);
    return TID_OK;
}

extern "C" int tid_server_get_stats(tid_server *S, tid_server_stats *out) {
    clear_error();
    if (!S || !out) return fail(TID_ERR_ARG, "tid_server_get_stats: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return TID_OK;
}

extern "C" int tid_server_destroy(tid_server *S) {
    clear_error();
    if (!S) return TID_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (int w = 0; w < S->cfg.workers; ++w)
        if (S->workers[w].th.joinable()) S->workers[w].th.join();
    destroy_workers(S);
    delete S;
    return TID_OK;
}
