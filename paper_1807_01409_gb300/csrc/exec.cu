// tid_exec: evaluate a subquery plan on the device (Section 4.3 and its figure
// "Integration of several operations": the query is split into subqueries,
// every subquery is searched against the TripleIDs and its matches extracted
// into a result vector -- with the filter applied during this step -- then the
// vectors are joined from left to right and the final results kept distinct).
//
//  * all MATCH nodes are searched together, up to 16 per multi-pattern pass
//    (the paper's keysArray: one scan marks every subquery a triple answers);
//  * a FILTER (or chain of FILTERs) that is the only reader of a MATCH is
//    folded into that MATCH's extraction pass;
//  * JOIN / UNION / PROJECT nodes run in node order (left-deep joins, as the
//    paper's REL list), each on the device; a node's result is freed after its
//    last reader has run.
#include <vector>

#include "ops.cuh"

namespace tid {
int pattern_vars(const tid_pattern &pat, int8_t *vars, int *k, bool *anonymous);
int bind_set(tid_ctx *ctx, const tid_store *st, const tid_pattern &pat, const tid_set *idx, const tid_pred *preds,
             int n_preds, tid_set **out);
}  // namespace tid

using namespace tid;

namespace {

int validate(const tid_plan_node *nodes, int n) {
    for (int i = 0; i < n; ++i) {
        const tid_plan_node &nd = nodes[i];
        int want_lo = 0, want_hi = 0;
        switch (nd.op) {
            case TID_OP_MATCH: want_lo = want_hi = 0; break;
            case TID_OP_FILTER:
            case TID_OP_PROJECT: want_lo = want_hi = 1; break;
            case TID_OP_JOIN: want_lo = want_hi = 2; break;
            case TID_OP_UNION: want_lo = 1; want_hi = 4; break;
            default: return fail(TID_ERR_ARG, "tid_exec: node %d has unknown op %d", i, nd.op);
        }
        if (nd.n_in < want_lo || nd.n_in > want_hi)
            return fail(TID_ERR_ARG, "tid_exec: node %d (op %d) has %d inputs", i, nd.op, nd.n_in);
        for (int j = 0; j < nd.n_in; ++j)
            if (nd.in[j] < 0 || nd.in[j] >= i)
                return fail(TID_ERR_ARG, "tid_exec: node %d reads node %d (must be earlier)", i, nd.in[j]);
    }
    return TID_OK;
}

}  // namespace

namespace tid {

int validate_plan(const tid_plan_node *nodes, int n_nodes) {
    if (n_nodes < 1) return fail(TID_ERR_ARG, "tid_exec: empty plan");
    TID_TRY(validate(nodes, n_nodes));
    for (int i = 0; i < n_nodes; ++i) {
        if (nodes[i].op == TID_OP_MATCH) {
            int8_t v[TID_MAX_COLS];
            int k = 0;
            bool anon = false;
            TID_TRY(pattern_vars(nodes[i].pattern, v, &k, &anon));
        }
        if (nodes[i].op == TID_OP_JOIN) {  // the algorithm and outer-join flags tid_join accepts
            const int a = nodes[i].algo, outer = a & (TID_JOIN_LEFT | TID_JOIN_RIGHT), base = a & ~outer;
            if ((base != TID_JOIN_AUTO && base != TID_JOIN_SORT_MERGE && base != TID_JOIN_HASH) ||
                (outer && base == TID_JOIN_HASH))
                return fail(TID_ERR_ARG, "tid_exec: node %d: join algorithm %d", i, a);
        }
    }
    return TID_OK;
}

// Evaluates a validated plan.  matched[i], for a MATCH node i, is its index list
// when the caller searched it already (taken over and freed here), or null.
int exec_plan(tid_ctx *ctx, const tid_store *st, const tid_plan_node *nodes, int n_nodes, tid_set **matched,
              tid_set **out) {
    *out = nullptr;

    std::vector<int> readers(n_nodes, 0);
    for (int i = 0; i < n_nodes; ++i)
        for (int j = 0; j < nodes[i].n_in; ++j) readers[nodes[i].in[j]]++;
    readers[n_nodes - 1]++;  // the result is read by the caller

    // fusion: FILTER chains that are the only reader of a MATCH
    std::vector<int> root(n_nodes, -1);
    std::vector<std::vector<tid_pred>> fused(n_nodes);
    for (int i = 0; i < n_nodes; ++i) {
        if (nodes[i].op == TID_OP_MATCH) {
            root[i] = i;
            continue;
        }
        if (nodes[i].op != TID_OP_FILTER) continue;
        const int in = nodes[i].in[0];
        const int r = root[in];
        if (r >= 0 && readers[in] == 1 && (int)fused[r].size() < TID_MAX_PREDS) {
            fused[r].push_back(nodes[i].pred);
            root[i] = r;
        }
    }

    std::vector<tid_set *> res(n_nodes, nullptr);
    std::vector<tid_set *> idx(n_nodes, nullptr);
    int rc = TID_OK;

    // 1) search: all MATCH nodes not searched yet, up to TID_MAX_MULTI per pass
    std::vector<int> matches;
    for (int i = 0; i < n_nodes; ++i) {
        if (nodes[i].op != TID_OP_MATCH) continue;
        if (matched && matched[i]) {
            idx[i] = matched[i];
            matched[i] = nullptr;
        } else {
            matches.push_back(i);
        }
    }
    for (size_t b = 0; b < matches.size() && rc == TID_OK; b += TID_MAX_MULTI) {
        const int m = (int)std::min<size_t>(TID_MAX_MULTI, matches.size() - b);
        tid_pattern pats[TID_MAX_MULTI];
        tid_set *outs[TID_MAX_MULTI];
        for (int j = 0; j < m; ++j) pats[j] = nodes[matches[b + j]].pattern;
        rc = m == 1 ? tid_match(ctx, st, pats[0], &outs[0]) : tid_match_multi(ctx, st, pats, m, outs);
        if (rc != TID_OK) break;
        for (int j = 0; j < m; ++j) idx[matches[b + j]] = outs[j];
    }

    auto release = [&](int i) {
        if (--readers[i] == 0 && res[i]) {
            set_free(res[i]);
            res[i] = nullptr;
        }
    };

    // 2) extraction and operators in node order
    for (int i = 0; i < n_nodes && rc == TID_OK; ++i) {
        const tid_plan_node &nd = nodes[i];
        switch (nd.op) {
            case TID_OP_MATCH:
                rc = bind_set(ctx, st, nd.pattern, idx[i], fused[i].data(), (int)fused[i].size(), &res[i]);
                set_free(idx[i]);
                idx[i] = nullptr;
                break;
            case TID_OP_FILTER:
                if (root[i] >= 0) {  // folded into the MATCH extraction: take over its result
                    res[i] = res[nd.in[0]];
                    res[nd.in[0]] = nullptr;
                    readers[nd.in[0]]--;
                } else {
                    rc = filter_set(ctx, res[nd.in[0]], &nd.pred, 1, &res[i]);
                    if (rc == TID_OK) release(nd.in[0]);
                }
                break;
            case TID_OP_JOIN:
                rc = join_sets(ctx, res[nd.in[0]], res[nd.in[1]], nd.algo, &res[i]);
                if (rc == TID_OK) {
                    release(nd.in[0]);
                    release(nd.in[1]);
                }
                break;
            case TID_OP_UNION: {
                const tid_set *ins[4];
                for (int j = 0; j < nd.n_in; ++j) ins[j] = res[nd.in[j]];
                rc = union_sets(ctx, ins, nd.n_in, &res[i]);
                if (rc == TID_OK)
                    for (int j = 0; j < nd.n_in; ++j) release(nd.in[j]);
                break;
            }
            case TID_OP_PROJECT:
                rc = project_set(ctx, res[nd.in[0]], nd.vars, nd.n_vars, &res[i]);
                if (rc == TID_OK) release(nd.in[0]);
                break;
        }
        if (rc == TID_OK && !res[i]) rc = fail(TID_ERR_ARG, "tid_exec: node %d produced nothing", i);
    }
    if (rc == TID_OK) {
        *out = res[n_nodes - 1];
        res[n_nodes - 1] = nullptr;
    }
    for (int i = 0; i < n_nodes; ++i) {
        if (res[i]) set_free(res[i]);
        if (idx[i]) set_free(idx[i]);
        if (matched && matched[i]) {
            set_free(matched[i]);
            matched[i] = nullptr;
        }
    }
    return rc;
}

}  // namespace tid

extern "C" int tid_plan_check(const tid_plan_node *nodes, int n_nodes) {
    clear_error();
    if (!nodes && n_nodes > 0) return fail(TID_ERR_ARG, "tid_plan_check: null plan");
    return validate_plan(nodes, n_nodes);
}

extern "C" int tid_exec(tid_ctx *ctx, const tid_store *st, const tid_plan_node *nodes, int n_nodes, tid_set **out) {
    clear_error();
    tid::Range nvtx_range("tid_exec");
    if (!ctx || !st || !nodes || !out) return fail(TID_ERR_ARG, "tid_exec: null argument");
    *out = nullptr;
    if (st->ctx != ctx) return fail(TID_ERR_ARG, "tid_exec: store belongs to another context");
    TID_TRY(validate_plan(nodes, n_nodes));
    DeviceGuard g(ctx->device);
    return exec_plan(ctx, st, nodes, n_nodes, nullptr, out);
}
