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
//     conclusion's terms kept with DISTINCT.
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
        uint32_t h = ((uint32_t)key * 0x9E3779B1u) >> (32 - tbits);
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
    // the distinct join terms among them (the paper's #Dist2)
    int kcol = 0;
    for (int c = 0; c < kb; ++c)
        if (bvars[c] == R.on) kcol = c;
    tid_set *K2 = nullptr;
    const int32_t *kcols[1] = {Braw->col[kcol]};
    TID_TRY(canonicalize(ctx, kcols, 1, &R.on, sx.res2, true, nullptr, &K2));
    hold.keep(K2);
    TID_TRY(rows_of(K2, &sx.dist2));
    B = Braw;  // rows in store order: the join below needs no order

    // 4) join on the shared term (the schema side is the small one: a hash join
    //    with it as the table, rows left in the order written), then the
    //    conclusion's variables put in canonical order with DISTINCT -- the one
    //    sort of the rule
    tid_set *J = nullptr, *C = nullptr;
    TID_TRY(join_sets(ctx, A, B, TID_JOIN_HASH, &J, false));
    hold.keep(J);
    int8_t cvars[3];
    int kc = 0;
    const int32_t *ccols[3];
    Bounds cb{};
    for (int slot = 0; slot < 3; ++slot)
        if (R.then_var[slot] >= 0) {
            int c = 0;
            while (J->vars[c] != R.then_var[slot]) ++c;
            ccols[kc] = J->col[c];
            cb.lo[kc] = J->lo[c];
            cb.hi[kc] = J->hi[c];
            cvars[kc++] = R.then_var[slot];
        }
    int64_t nj = 0;
    TID_TRY(rows_of(J, &nj));
    TID_TRY(canonicalize(ctx, ccols, kc, cvars, nj, true, J->bounded ? &cb : nullptr, &C));
    hold.keep(C);
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
