// Internal interfaces of the tuple-set operators (bind, filter, sort, join,
// union, project) shared by the translation units.
#pragma once

#include "tid_internal.cuh"

namespace tid {

constexpr int MAX_PREDS = 4;  // predicates fused into one compaction pass

struct Pred {  // a FILTER predicate on column `col` of the set being produced
    int col;
    int op;
    int32_t a, b;
};

struct OutCols {
    int32_t *col[TID_MAX_COLS];
};

// Rows of k int32 columns packed into one unsigned key: field c holds
// order_key(col_c) - min[c] (order_key flips the sign bit, so unsigned order is
// int32 order) in bits [shift[c], shift[c] + width); column 0 is the most
// significant field, so key order is row order.
struct PackSpec {
    uint32_t min[TID_MAX_COLS];
    uint32_t shift[TID_MAX_COLS];
    unsigned long long mask[TID_MAX_COLS];
};

// Column value bounds in sort order (int32 ^ 0x80000000); any valid bounds
// serve the packed sort, exact ones make its keys narrowest.
struct Bounds {
    uint32_t lo[TID_MAX_COLS], hi[TID_MAX_COLS];
};

// exclusive scan of n uint32 (out may alias in); *total_dev receives the sum
int scan_exclusive_u32(tid_ctx *ctx, const uint32_t *in, uint32_t *out, int64_t n,
                       unsigned long long *total_dev);

// single-pass compactions (compact.cu); `out` must have capacity >= n
// bind; if mm is not null, mm[c] / mm[8 + c] receive (atomic min / max) the
// sort-order bounds of output column c over the kept rows (caller presets them)
int compact_bind(tid_ctx *ctx, const tid_store *st, const tid_pattern &pat, const int32_t *idx, int64_t n,
                 const Pred *preds, int n_preds, tid_set *out, uint32_t *mm);
int compact_filter(tid_ctx *ctx, const tid_set *in, int64_t n, const Pred *preds, int n_preds, tid_set *out);
// store triples (in store order) whose fixed_slot holds fixed_val (fixed_slot -1:
// any) and whose key_slot term is in the key table (2^tbits slots, home slot =
// top tbits bits of key * 0x9E3779B1, linear probing, 0 = empty); output column
// c = slot src[c]
int compact_semijoin(tid_ctx *ctx, const tid_store *st, int fixed_slot, int32_t fixed_val, int key_slot,
                     const int32_t *table, int tbits, const int8_t *src, tid_set *out);
int compact_unique(tid_ctx *ctx, const int32_t *const *cols, int k, const int32_t *perm, int64_t n,
                   tid_set *out);
// sorted packed keys (64-bit if wide, else 32-bit) -> distinct rows of k columns
int compact_unique_packed(tid_ctx *ctx, const void *keys, bool wide, int k, int64_t n, const PackSpec &ps,
                          tid_set *out);

// sorting (sort.cu)
// perm receives the stable permutation that orders rows 0..n-1 lexicographically
// by the key columns keys[0..nk-1] (signed int32 order).
int sort_perm(tid_ctx *ctx, const int32_t *const *keys, int nk, int64_t n, int32_t *perm);
// out[c][i] = in[c][perm[i]] for c < k, i < n
int gather_cols(tid_ctx *ctx, const int32_t *const *in, int k, const int32_t *perm, int64_t n,
                int32_t *const *out);
// canonical form (rows sorted in column order; duplicates dropped if dedupe);
// bounds of the input columns if known (else they are computed); the output
// set records the bounds used
// sorted_tail: the rows are already sorted by their last sorted_tail columns
// (lexicographically, in that order), so only the leading columns are sorted
int canonicalize(tid_ctx *ctx, const int32_t *const *cols, int k, const int8_t *vars, int64_t n,
                 bool dedupe, const Bounds *bounds, tid_set **out, int sorted_tail = 0);

// write a known row count into a set (device count and host mirror)
int set_rows_const(tid_set *set, int64_t n);

// row count known on the host (waits for the producer if needed)
int set_rows_host(tid_set *set, int64_t *rows);
int set_rows_host(const tid_set *set, int64_t *rows);

// joins (join.cu); right and full outer joins composed from the left join (ops.cu)
// sorted_out = false (internal use, hash join of inputs in any row order): the
// joined rows in the order written, not canonical (the caller sorts what it keeps)
int join_sets(tid_ctx *ctx, const tid_set *L, const tid_set *R, int algo, tid_set **out, bool sorted_out = true);
int outer_join_sets(tid_ctx *ctx, const tid_set *L, const tid_set *R, int algo, tid_set **out);

// merge (merge.cu): the distinct rows of two sets each sorted in the same nu
// columns (acols / bcols, null = absent column, read as 0) into out (capacity
// >= na + nb), in order; writes the row count
int merge_unique(tid_ctx *ctx, const int32_t *const *acols, int64_t na, const int32_t *const *bcols, int64_t nb,
                 int nu, tid_set *out);

// set operators (ops.cu)
int filter_set(tid_ctx *ctx, const tid_set *in, const tid_pred *preds, int n_preds, tid_set **out);
int union_sets(tid_ctx *ctx, const tid_set *const *in, int k, tid_set **out);
int project_set(tid_ctx *ctx, const tid_set *in, const int8_t *vars, int n_vars, tid_set **out);

// plans (exec.cu): checks a plan's shape and patterns; evaluates a checked plan,
// taking over matched[i] (an index list, or null to search it) for MATCH nodes
int validate_plan(const tid_plan_node *nodes, int n_nodes);
int exec_plan(tid_ctx *ctx, const tid_store *st, const tid_plan_node *nodes, int n_nodes, tid_set **matched,
              tid_set **out);

}  // namespace tid
