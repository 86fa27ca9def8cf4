// C ABI of the tuple-set operators (Section 4): bind (result vectors of a
// subquery, with fused filters), filter, join, union, project, and sets
// imported from host memory.
#include <string.h>

#include <algorithm>

#include <vector>

#include "ops.cuh"

namespace tid {

int set_rows_const(tid_set *set, int64_t n);

namespace {

bool valid_var(int v) { return v >= 0 && v <= 127; }

int find_col(const tid_set *s, int var) {
    for (int c = 0; c < s->k; ++c)
        if (s->vars[c] == var) return c;
    return -1;
}

int make_preds(const int8_t *vars, int k, const tid_pred *preds, int n_preds, Pred *out, const char *who) {
    if (n_preds < 0 || n_preds > MAX_PREDS) return fail(TID_ERR_ARG, "%s: %d predicates (max %d)", who, n_preds, MAX_PREDS);
    if (n_preds > 0 && !preds) return fail(TID_ERR_ARG, "%s: null predicates", who);
    for (int q = 0; q < n_preds; ++q) {
        int col = -1;
        for (int c = 0; c < k; ++c)
            if (vars[c] == preds[q].var) col = c;
        if (col < 0) return fail(TID_ERR_ARG, "%s: predicate on variable %d not in the set", who, preds[q].var);
        if (preds[q].op < TID_CMP_EQ || preds[q].op > TID_CMP_RANGE)
            return fail(TID_ERR_ARG, "%s: unknown comparison %d", who, preds[q].op);
        out[q] = Pred{col, preds[q].op, preds[q].a, preds[q].b};
    }
    return TID_OK;
}

int empty_set(tid_ctx *ctx, int k, const int8_t *vars, tid_set **out) {
    tid_set *e = nullptr;
    TID_TRY(set_alloc(ctx, k, vars, 0, &e));
    int rc = set_rows_const(e, 0);
    if (rc == TID_OK) rc = set_ready(e);
    if (rc != TID_OK) {
        set_free(e);
        return rc;
    }
    *out = e;
    return TID_OK;
}

}  // namespace

// output variables of a pattern: distinct ids at its "?" slots in slot order
int pattern_vars(const tid_pattern &pat, int8_t *vars, int *k, bool *anonymous) {
    const int32_t key[3] = {pat.s, pat.p, pat.o};
    *k = 0;
    *anonymous = false;
    for (int j = 0; j < 3; ++j) {
        const int v = pat.var[j];
        if (key[j] < 0) return fail(TID_ERR_ID, "negative ID in pattern");
        if (v >= 0) {
            if (key[j] != 0) return fail(TID_ERR_ARG, "bound slot %d carries variable %d", j, v);
            if (!valid_var(v)) return fail(TID_ERR_ARG, "variable id %d out of range", v);
            bool seen = false;
            for (int c = 0; c < *k; ++c) seen = seen || vars[c] == v;
            if (!seen) vars[(*k)++] = (int8_t)v;
        } else if (key[j] == 0) {
            *anonymous = true;
        }
    }
    if (*k == 0) return fail(TID_ERR_ARG, "pattern has no variable");
    return TID_OK;
}

int bind_set(tid_ctx *ctx, const tid_store *st, const tid_pattern &pat, const tid_set *idx, const tid_pred *preds,
             int n_preds, tid_set **out) {
    int8_t vars[TID_MAX_COLS];
    int k = 0;
    bool anon = false;
    TID_TRY(pattern_vars(pat, vars, &k, &anon));
    Pred pr[MAX_PREDS];
    TID_TRY(make_preds(vars, k, preds, n_preds, pr, "tid_bind"));
    int64_t n = 0;
    TID_TRY(set_rows_host(idx, &n));
    if (n == 0) return empty_set(ctx, k, vars, out);
    tid_set *tmp = nullptr;
    TID_TRY(set_alloc(ctx, k, vars, n, &tmp));
    uint32_t *mm = nullptr;  // column bounds of the extracted rows, for the sort
    int rc = dev_alloc(ctx, (void **)&mm, 2 * TID_MAX_COLS * sizeof(uint32_t));
    if (rc == TID_OK) {
        cudaError_t e = cudaMemsetAsync(mm, 0xFF, TID_MAX_COLS * sizeof(uint32_t), ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(mm + TID_MAX_COLS, 0, TID_MAX_COLS * sizeof(uint32_t), ctx->stream);
        if (e != cudaSuccess) rc = fail_cuda(e, "tid_bind");
    }
    if (rc == TID_OK) rc = compact_bind(ctx, st, pat, idx->col[0], n, pr, n_preds, tmp, mm);
    uint32_t hb[2 * TID_MAX_COLS];
    if (rc == TID_OK) {
        cudaError_t e = cudaMemcpyAsync(hb, mm, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) rc = fail_cuda(e, "tid_bind bounds");
    }
    if (rc == TID_OK) rc = set_ready(tmp);
    int64_t m = 0;
    if (rc == TID_OK) rc = set_rows_host(tmp, &m);
    const int32_t *cols[TID_MAX_COLS];
    Bounds b{};
    for (int c = 0; c < k; ++c) {
        cols[c] = tmp->col[c];
        b.lo[c] = hb[c];
        b.hi[c] = hb[TID_MAX_COLS + c];
    }
    // In a store sorted by (s, p, o) the hits, in index order, are sorted by
    // their variable slots in slot order (the bound slots are constant) when
    // no anonymous slot comes before a variable -- the set's canonical order.
    // The compaction keeps index order, so no sort is needed: the rows are
    // the result, or (an anonymous slot last) one pass drops adjacent repeats.
    bool in_order = rc == TID_OK;
    {
        const int32_t key[3] = {pat.s, pat.p, pat.o};
        bool seen_anon = false;
        for (int j = 0; j < 3; ++j) {
            if (pat.var[j] >= 0) in_order = in_order && !seen_anon;
            else if (key[j] == 0) seen_anon = true;
        }
    }
    if (in_order) in_order = store_spo_sorted(st);
    if (in_order && !anon) {
        tmp->bounded = m > 0;
        for (int c = 0; c < k; ++c) {
            tmp->lo[c] = b.lo[c];
            tmp->hi[c] = b.hi[c];
        }
        if (mm) dev_free(ctx, mm);
        *out = tmp;
        return TID_OK;
    }
    if (in_order) {
        tid_set *o = nullptr;
        const int32_t *none[TID_MAX_COLS] = {nullptr};
        rc = set_alloc(ctx, k, vars, m, &o);
        if (rc == TID_OK) rc = merge_unique(ctx, cols, m, none, 0, k, o);
        if (rc == TID_OK) rc = set_ready(o);
        if (rc == TID_OK) {
            o->bounded = m > 0;
            for (int c = 0; c < k; ++c) {
                o->lo[c] = b.lo[c];
                o->hi[c] = b.hi[c];
            }
            *out = o;
        } else if (o) {
            set_free(o);
        }
    } else if (rc == TID_OK) {
        // distinct triples give distinct rows unless a "?" slot is anonymous
        rc = canonicalize(ctx, cols, k, vars, m, anon, &b, out);
    }
    if (mm) dev_free(ctx, mm);
    set_free(tmp);
    return rc;
}

int filter_set(tid_ctx *ctx, const tid_set *in, const tid_pred *preds, int n_preds, tid_set **out) {
    Pred pr[MAX_PREDS];
    TID_TRY(make_preds(in->vars, in->k, preds, n_preds, pr, "tid_filter"));
    int64_t n = 0;
    TID_TRY(set_rows_host(in, &n));
    tid_set *o = nullptr;
    TID_TRY(set_alloc(ctx, in->k, in->vars, n, &o));
    int rc = compact_filter(ctx, in, n, pr, n_preds, o);
    if (rc == TID_OK) rc = set_ready(o);
    if (rc == TID_OK && in->bounded) {  // a subset keeps its input's bounds
        o->bounded = true;
        for (int c = 0; c < in->k; ++c) {
            o->lo[c] = in->lo[c];
            o->hi[c] = in->hi[c];
        }
    }
    if (rc != TID_OK) {
        set_free(o);
        return rc;
    }
    *out = o;
    return TID_OK;
}

int union_sets(tid_ctx *ctx, const tid_set *const *in, int k, tid_set **out) {
    if (k < 1 || !in) return fail(TID_ERR_ARG, "tid_union: need at least one set");
    int8_t uv[TID_MAX_COLS];
    int nu = 0;
    int64_t total = 0;
    std::vector<int64_t> rows(k);
    for (int i = 0; i < k; ++i) {
        if (!in[i] || in[i]->ctx != ctx) return fail(TID_ERR_ARG, "tid_union: bad input %d", i);
        for (int c = 0; c < in[i]->k; ++c) {
            bool seen = false;
            for (int u = 0; u < nu; ++u) seen = seen || uv[u] == in[i]->vars[c];
            if (!seen) {
                if (nu == TID_MAX_COLS) return fail(TID_ERR_ARG, "tid_union: more than %d variables", TID_MAX_COLS);
                uv[nu++] = in[i]->vars[c];
            }
        }
        TID_TRY(set_rows_host(in[i], &rows[i]));
        total += rows[i];
    }
    if (total > INT32_MAX) return fail(TID_ERR_CAPACITY, "tid_union: %lld rows", (long long)total);
    // bounds of the union: each input's bounds, or the padding value 0
    Bounds b{};
    bool known = true;
    for (int u = 0; u < nu; ++u) {
        b.lo[u] = 0xFFFFFFFFu;
        b.hi[u] = 0u;
    }
    for (int i = 0; i < k && known; ++i) {
        if (rows[i] == 0) continue;
        if (!in[i]->bounded) {
            known = false;
            break;
        }
        for (int u = 0; u < nu; ++u) {
            const int c = find_col(in[i], uv[u]);
            const uint32_t lo = c >= 0 ? in[i]->lo[c] : 0x80000000u;
            const uint32_t hi = c >= 0 ? in[i]->hi[c] : 0x80000000u;
            b.lo[u] = std::min(b.lo[u], lo);
            b.hi[u] = std::max(b.hi[u], hi);
        }
    }
    // Each input is canonical in its own column order; padded to the union
    // schema it stays sorted when its columns keep their relative order there
    // (a constant 0 column never reorders rows).  Then the union is a chain of
    // merges that drop duplicates, with no sort.
    bool ordered = true;
    for (int i = 0; i < k && ordered; ++i) {
        int last = -1;
        for (int u = 0; u < nu; ++u) {
            const int c = find_col(in[i], uv[u]);
            if (c < 0) continue;
            ordered = ordered && c > last;
            last = c;
        }
    }
    if (ordered) {
        tid_set *cur = nullptr;  // union of the inputs merged so far (null: only in[0])
        int rc = TID_OK;
        for (int i = 1; i < k && rc == TID_OK; ++i) {
            const int32_t *ac[TID_MAX_COLS], *bc[TID_MAX_COLS];
            const tid_set *A = cur ? cur : in[0];
            for (int u = 0; u < nu; ++u) {
                const int ca = find_col(A, uv[u]), cb = find_col(in[i], uv[u]);
                ac[u] = ca >= 0 ? A->col[ca] : nullptr;
                bc[u] = cb >= 0 ? in[i]->col[cb] : nullptr;
            }
            int64_t na = 0;
            rc = set_rows_host(A, &na);
            tid_set *m = nullptr;
            if (rc == TID_OK) rc = set_alloc(ctx, nu, uv, na + rows[i], &m);
            if (rc == TID_OK) rc = merge_unique(ctx, ac, na, bc, rows[i], nu, m);
            if (rc == TID_OK) rc = set_ready(m);
            if (cur) set_free(cur);
            cur = m;
            if (rc != TID_OK) {
                if (cur) set_free(cur);
                return rc;
            }
        }
        if (!cur) {  // one input: its rows in the union schema (already canonical)
            const int32_t *ac[TID_MAX_COLS], *none[TID_MAX_COLS] = {nullptr};
            for (int u = 0; u < nu; ++u) ac[u] = in[0]->col[find_col(in[0], uv[u])];
            rc = set_alloc(ctx, nu, uv, rows[0], &cur);
            if (rc == TID_OK) rc = merge_unique(ctx, ac, rows[0], none, 0, nu, cur);
            if (rc == TID_OK) rc = set_ready(cur);
            if (rc != TID_OK) {
                if (cur) set_free(cur);
                return rc;
            }
        }
        cur->bounded = known && total > 0;
        for (int u = 0; u < nu && cur->bounded; ++u) {
            cur->lo[u] = b.lo[u];
            cur->hi[u] = b.hi[u];
        }
        *out = cur;
        return TID_OK;
    }
    // otherwise: concatenate in the union schema (absent variables = 0), then canonical form
    void *block = nullptr;
    const size_t colb = ((size_t)(total > 0 ? total : 1) * 4 + 255) / 256 * 256;
    TID_TRY(dev_alloc(ctx, &block, colb * nu));
    int rc = TID_OK;
    int64_t at = 0;
    const int32_t *cols[TID_MAX_COLS];
    for (int u = 0; u < nu; ++u) cols[u] = (const int32_t *)((char *)block + colb * u);
    for (int i = 0; i < k && rc == TID_OK; ++i) {
        if (rows[i] == 0) continue;
        for (int u = 0; u < nu && rc == TID_OK; ++u) {
            int32_t *dst = (int32_t *)cols[u] + at;
            const int c = find_col(in[i], uv[u]);
            cudaError_t e = c >= 0 ? cudaMemcpyAsync(dst, in[i]->col[c], (size_t)rows[i] * 4, cudaMemcpyDeviceToDevice, ctx->stream)
                                   : cudaMemsetAsync(dst, 0, (size_t)rows[i] * 4, ctx->stream);
            if (e != cudaSuccess) rc = fail_cuda(e, "tid_union copy");
        }
        at += rows[i];
    }
    if (rc == TID_OK) rc = canonicalize(ctx, cols, nu, uv, total, true, known && total > 0 ? &b : nullptr, out);
    dev_free(ctx, block);
    return rc;
}

int project_set(tid_ctx *ctx, const tid_set *in, const int8_t *vars, int n_vars, tid_set **out) {
    if (n_vars < 1 || n_vars > TID_MAX_COLS || !vars) return fail(TID_ERR_ARG, "tid_project: %d variables", n_vars);
    const int32_t *cols[TID_MAX_COLS];
    for (int i = 0; i < n_vars; ++i) {
        for (int j = 0; j < i; ++j)
            if (vars[j] == vars[i]) return fail(TID_ERR_ARG, "tid_project: variable %d twice", vars[i]);
        const int c = find_col(in, vars[i]);
        if (c < 0) return fail(TID_ERR_ARG, "tid_project: variable %d not in the set", vars[i]);
        cols[i] = in->col[c];
    }
    int64_t n = 0;
    TID_TRY(set_rows_host(in, &n));
    // keeping all columns in order of a canonical input is the identity
    bool identity = n_vars == in->k;
    for (int i = 0; i < n_vars && identity; ++i) identity = in->vars[i] == vars[i];
    Bounds b{};
    for (int i = 0; i < n_vars; ++i) {
        const int c = find_col(in, vars[i]);
        b.lo[i] = in->lo[c];
        b.hi[i] = in->hi[c];
    }
    // a leading prefix of a canonical set's columns is sorted already, its
    // duplicates adjacent: one pass drops them
    bool prefix = !identity;
    for (int i = 0; i < n_vars && prefix; ++i) prefix = in->vars[i] == vars[i];
    if (prefix) {
        tid_set *o = nullptr;
        const int32_t *none[TID_MAX_COLS] = {nullptr};
        TID_TRY(set_alloc(ctx, n_vars, vars, n, &o));
        int rc = merge_unique(ctx, cols, n, none, 0, n_vars, o);
        if (rc == TID_OK) rc = set_ready(o);
        if (rc != TID_OK) {
            set_free(o);
            return rc;
        }
        o->bounded = in->bounded;
        for (int i = 0; i < n_vars && o->bounded; ++i) {
            o->lo[i] = b.lo[i];
            o->hi[i] = b.hi[i];
        }
        *out = o;
        return TID_OK;
    }
    // The input is sorted by its leading columns; when the requested order ends
    // with them (e.g. (x, v) -> (v, x)) the rows are already in order of that
    // tail and only the leading requested columns need sorting.
    int tail = 0;
    for (int t = n_vars; t >= 1 && tail == 0; --t) {
        bool ok = true;
        for (int i = 0; i < t && ok; ++i) ok = in->vars[i] == vars[n_vars - t + i];
        if (ok) tail = t;
    }
    return canonicalize(ctx, cols, n_vars, vars, n, !identity, in->bounded ? &b : nullptr, out, tail);
}

// Right and full outer joins (Section 4.2 lists the outer joins of the library
// the paper used) from the left join: right(L, R) keeps every row of R -- it is
// the left join of R with L, its columns put in the join's order (L's, then R's
// others) -- and full(L, R) is the union of left(L, R) and right(L, R), whose
// matched rows are the same tuples and are kept once.
int outer_join_sets(tid_ctx *ctx, const tid_set *L, const tid_set *R, int algo, tid_set **out) {
    *out = nullptr;
    const int base = algo & ~(TID_JOIN_LEFT | TID_JOIN_RIGHT);
    if (base != TID_JOIN_AUTO && base != TID_JOIN_SORT_MERGE)
        return fail(TID_ERR_ARG, "tid_join: outer joins run as sort-merge joins (algo %d)", algo);
    int8_t ovars[TID_MAX_COLS];
    int k = 0;
    for (int c = 0; c < L->k; ++c) ovars[k++] = L->vars[c];
    for (int d = 0; d < R->k; ++d) {
        bool shared = false;
        for (int c = 0; c < L->k; ++c) shared = shared || L->vars[c] == R->vars[d];
        if (shared) continue;
        if (k == TID_MAX_COLS) return fail(TID_ERR_ARG, "tid_join: output wider than %d columns", TID_MAX_COLS);
        ovars[k++] = R->vars[d];
    }
    tid_set *rl = nullptr, *right = nullptr;
    TID_TRY(join_sets(ctx, R, L, TID_JOIN_LEFT | base, &rl));
    int rc = project_set(ctx, rl, ovars, k, &right);
    set_free(rl);
    TID_TRY(rc);
    if (!(algo & TID_JOIN_LEFT)) {
        *out = right;
        return TID_OK;
    }
    tid_set *lj = nullptr;
    rc = join_sets(ctx, L, R, TID_JOIN_LEFT | base, &lj);
    if (rc == TID_OK) {
        const tid_set *both[2] = {lj, right};
        rc = union_sets(ctx, both, 2, out);
    }
    set_free(lj);
    set_free(right);
    return rc;
}

}  // namespace tid

using namespace tid;

static int check_set(const tid_ctx *ctx, const tid_set *s, const char *who) {
    if (!s) return fail(TID_ERR_ARG, "%s: null set", who);
    if (s->ctx != ctx) return fail(TID_ERR_ARG, "%s: set belongs to another context", who);
    return TID_OK;
}

extern "C" int tid_bind(tid_ctx *ctx, const tid_store *st, tid_pattern pat, const tid_set *idx, const tid_pred *preds,
                        int n_preds, tid_set **out) {
    clear_error();
    tid::Range nvtx_range("tid_bind");
    if (!ctx || !st || !out) return fail(TID_ERR_ARG, "tid_bind: null argument");
    *out = nullptr;
    TID_TRY(check_set(ctx, idx, "tid_bind"));
    if (st->ctx != ctx) return fail(TID_ERR_ARG, "tid_bind: store belongs to another context");
    if (idx->k != 1 || idx->vars[0] != -1) return fail(TID_ERR_ARG, "tid_bind: idx must be an index set from tid_match");
    DeviceGuard g(ctx->device);
    return bind_set(ctx, st, pat, idx, preds, n_preds, out);
}

extern "C" int tid_filter(tid_ctx *ctx, const tid_set *in, const tid_pred *preds, int n_preds, tid_set **out) {
    clear_error();
    tid::Range nvtx_range("tid_filter");
    if (!ctx || !out) return fail(TID_ERR_ARG, "tid_filter: null argument");
    *out = nullptr;
    TID_TRY(check_set(ctx, in, "tid_filter"));
    DeviceGuard g(ctx->device);
    return filter_set(ctx, in, preds, n_preds, out);
}

extern "C" int tid_join(tid_ctx *ctx, const tid_set *L, const tid_set *R, int algo, tid_set **out) {
    clear_error();
    tid::Range nvtx_range("tid_join");
    if (!ctx || !out) return fail(TID_ERR_ARG, "tid_join: null argument");
    *out = nullptr;
    TID_TRY(check_set(ctx, L, "tid_join"));
    TID_TRY(check_set(ctx, R, "tid_join"));
    DeviceGuard g(ctx->device);
    return join_sets(ctx, L, R, algo, out);
}

extern "C" int tid_union(tid_ctx *ctx, const tid_set *const *in, int k, tid_set **out) {
    clear_error();
    tid::Range nvtx_range("tid_union");
    if (!ctx || !out) return fail(TID_ERR_ARG, "tid_union: null argument");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    return union_sets(ctx, in, k, out);
}

extern "C" int tid_project(tid_ctx *ctx, const tid_set *in, const int8_t *vars, int n_vars, tid_set **out) {
    clear_error();
    tid::Range nvtx_range("tid_project");
    if (!ctx || !out) return fail(TID_ERR_ARG, "tid_project: null argument");
    *out = nullptr;
    TID_TRY(check_set(ctx, in, "tid_project"));
    DeviceGuard g(ctx->device);
    return project_set(ctx, in, vars, n_vars, out);
}

extern "C" int tid_set_from_host(tid_ctx *ctx, const int32_t *buf, int64_t rows, int cols, const int8_t *vars,
                                 tid_set **out) {
    clear_error();
    tid::Range nvtx_range("tid_set_from_host");
    if (!ctx || !out || !vars) return fail(TID_ERR_ARG, "tid_set_from_host: null argument");
    *out = nullptr;
    if (cols < 1 || cols > TID_MAX_COLS) return fail(TID_ERR_ARG, "tid_set_from_host: %d columns", cols);
    if (rows < 0 || rows > INT32_MAX) return fail(TID_ERR_ARG, "tid_set_from_host: %lld rows", (long long)rows);
    if (rows > 0 && !buf) return fail(TID_ERR_ARG, "tid_set_from_host: null buffer");
    for (int c = 0; c < cols; ++c) {
        if (!valid_var(vars[c])) return fail(TID_ERR_ARG, "tid_set_from_host: variable id %d", vars[c]);
        for (int d = 0; d < c; ++d)
            if (vars[d] == vars[c]) return fail(TID_ERR_ARG, "tid_set_from_host: variable %d twice", vars[c]);
    }
    DeviceGuard g(ctx->device);
    if (rows == 0) return empty_set(ctx, cols, vars, out);
    // transpose on the host, one copy per column
    std::vector<int32_t> colbuf((size_t)rows * cols);
    for (int64_t r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) colbuf[(size_t)c * rows + r] = buf[r * cols + c];
    void *block = nullptr;
    TID_TRY(dev_alloc(ctx, &block, colbuf.size() * 4));
    int rc = TID_OK;
    cudaError_t e = cudaMemcpyAsync(block, colbuf.data(), colbuf.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) rc = fail_cuda(e, "tid_set_from_host copy");
    if (rc == TID_OK) {
        const int32_t *cp[TID_MAX_COLS];
        for (int c = 0; c < cols; ++c) cp[c] = (const int32_t *)block + (size_t)c * rows;
        rc = canonicalize(ctx, cp, cols, vars, rows, true, nullptr, out);
        if (rc == TID_OK) rc = set_rows_host(*out, &rows);  // colbuf must outlive the copy
    }
    dev_free(ctx, block);
    return rc;
}
