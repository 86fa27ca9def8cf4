/*
 * tid.h -- C ABI of the GB300 TripleID-Q hot path (libtid.so).
 *
 * TripleID-Q (Chantrapornchai & Choksuchat, IEEE TPDS 2018) keeps an RDF graph
 * as dictionary-encoded triples of 32-bit IDs and answers triple patterns by a
 * brute-force data-parallel scan (Section 3, Algorithm 1), then combines the
 * per-pattern results with union, join and filter (Section 4).  This library
 * is that hot path on one GPU: the store is resident in device memory as three
 * int32 columns (structure of arrays), patterns are matched by a single-pass
 * scan-and-compact kernel, and the results are tuple sets consumed by join,
 * union, filter and projection kernels.
 *
 * Conventions
 *  - IDs are int32 >= 1.  The value 0 in a pattern is the free variable "?"
 *    (Section 3: the key encoding reserves 0 for "?").  In a tuple set 0 means
 *    "unbound" (a variable missing from one branch of a union); it never joins
 *    and never passes a filter.
 *  - A triple index is int32 in [0, n).  n <= 2^31 - 1.
 *  - A tuple set has k <= TID_MAX_COLS int32 columns, each labelled with a
 *    variable id (0..127), or, for the index sets returned by the match calls,
 *    a single column labelled -1.  Columns live in device memory (SoA).
 *  - Every call is ordered on the context's CUDA stream.  Calls that need a
 *    result size on the host (tid_join, tid_set_rows, tid_set_to_host, the
 *    plan executor) synchronise with that stream; the others do not.
 *  - Status: every call returns TID_OK or one of the TID_ERR_* codes below,
 *    and sets a thread-local message readable with tid_last_error().  No call
 *    aborts the process and no kernel traps: waits inside kernels give up
 *    after a bounded number of polls and report TID_ERR_TIMEOUT.
 *  - Ownership: the library owns every tid_ctx, tid_store and tid_set and the
 *    device memory behind them (stream-ordered allocations from a pool private
 *    to the context).  Free every store and set before destroying its context.
 */
#ifndef TID_H_
#define TID_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TID_OK            0
#define TID_ERR_ARG       1  /* null pointer, bad size, column, variable or op */
#define TID_ERR_ID        2  /* a negative ID in a pattern */
#define TID_ERR_OOM       3  /* device or pinned host allocation failed */
#define TID_ERR_CAPACITY  4  /* a caller buffer is too small; *needed holds the size */
#define TID_ERR_TIMEOUT   5  /* a bounded in-kernel wait gave up */
#define TID_ERR_CUDA      6  /* any other CUDA runtime error */

/* where the columns handed to tid_load live */
#define TID_HOST   0
#define TID_DEVICE 1

#define TID_MAX_COLS  8
#define TID_MAX_MULTI 16

typedef struct tid_ctx tid_ctx;
typedef struct tid_store tid_store;
typedef struct tid_set tid_set;

/*
 * A triple pattern (Section 3: "key.subj, key.pred, key.obj"; 0 = "?").
 * var[j] labels the "?" in slot j (0 = s, 1 = p, 2 = o) with a variable id
 * 0..127, or is -1 for an anonymous "?".  A bound slot (value != 0) must have
 * var[j] == -1.  The same variable in two slots (e.g. ?x p ?x) means the two
 * terms must be equal.  var[] is read only by the calls that build tuples.
 */
typedef struct {
    int32_t s, p, o;
    int8_t var[3];
    int8_t reserved; /* set to 0 */
} tid_pattern;

/* ------------------------------------------------------------------------ */
/* context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * owned by the caller (it must outlive the context), or NULL for a stream the
 * context creates and owns.  On success *out receives the context.  A process
 * drives one GPU (launch shapes are worked out once per process): a context
 * on another device than the first one any call of the process used fails
 * with TID_ERR_ARG.  Run one process per GPU. */
int tid_ctx_create(int device, void *cuda_stream, tid_ctx **out);

/* Wait for all work on the context's stream; returns TID_ERR_TIMEOUT if an
 * in-kernel wait gave up since the last check, TID_ERR_CUDA on a CUDA error. */
int tid_ctx_sync(tid_ctx *ctx);

/* Destroy the context (synchronises first).  NULL is accepted. */
int tid_ctx_destroy(tid_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *tid_last_error(void);

/* Testing aid for failure handling (the paper has no counterpart): after
 * `after` more device allocations on this context succeed, every further one
 * fails with TID_ERR_OOM as if the device were out of memory; after < 0 turns
 * it off.  The failure is made on the host (no allocation is attempted); calls
 * that fail this way release what they allocated and leave the context
 * usable. */
int tid_ctx_inject_alloc_failure(tid_ctx *ctx, int64_t after);

/* Testing aid for failure detection (the paper has no counterpart): runs on
 * the context stream one CTA that waits, with the library's bounded in-kernel
 * wait, at a barrier no other CTA reaches; after `polls` polls (1 .. 2^21) it
 * gives up and sets the context's error word, as a stalled look-back or grid
 * barrier would.  Synchronises and returns what the context then reports:
 * TID_ERR_TIMEOUT (reported once; the context stays usable).  TID_ERR_ARG for
 * polls out of range. */
int tid_ctx_test_bounded_wait(tid_ctx *ctx, int64_t polls);

/* ------------------------------------------------------------------------ */
/* store -- Section 3: the TripleID file of (SubjID, PredID, ObjID)          */
/* ------------------------------------------------------------------------ */

/* Make a store of n triples from three int32 columns s[i], p[i], o[i].
 *  where = TID_HOST:   host arrays (pageable or pinned); they are copied.
 *  where = TID_DEVICE: device arrays; copy = 1 copies them, copy = 0 borrows
 *                      them (no copy; they must stay valid and unchanged
 *                      while the store lives).
 * n may be 0.  IDs are not scanned for validity (an ID <= 0 in the store can
 * only ever be matched by "?").  The store must be a set (no repeated triple)
 * for the tuple-set calls to return sets.  One read of the store checks
 * whether its triples are in (s, p, o) order; tid_bind on such a store skips
 * its sort when index order is already the result's order.  Returns after the
 * copies and the check are queued on the context stream. */
int tid_load(tid_ctx *ctx, const int32_t *s, const int32_t *p, const int32_t *o,
             int64_t n, int where, int copy, tid_store **out);

/* Number of triples and the device columns of a store. */
int tid_store_info(const tid_store *st, int64_t *n, const int32_t **s,
                   const int32_t **p, const int32_t **o);

/* Free a store (NULL accepted).  Its own copy of the columns is released
 * stream-ordered on the context stream, so work already queued there that
 * reads it finishes first; borrowed columns are left to their owner.  Sets
 * made from the store hold their own memory and stay valid. */
int tid_store_free(tid_store *st);

/* ------------------------------------------------------------------------ */
/* search -- Section 3, Algorithm 1 (GPUSearch)                              */
/* ------------------------------------------------------------------------ */

/* All positions i whose triple answers the pattern, i.e.
 *   (p.s == 0 || S[i] == p.s) && (p.p == 0 || P[i] == p.p) && (p.o == 0 || O[i] == p.o),
 * as an ascending list of int32 indices: a one-column set labelled -1
 * (the paper's positionArray, compacted).  Only the bound columns are read.
 * Errors: TID_ERR_ID if a pattern value is negative.  Does not synchronise. */
int tid_match(tid_ctx *ctx, const tid_store *st, tid_pattern pat, tid_set **out);

/* Several patterns in ONE pass over the store (Section 4.1: the key array
 * holds the keys of all subqueries and every triple is marked with each
 * subquery it answers; one triple may answer several).  outs[j] receives the
 * ascending index list of pats[j], exactly as tid_match(pats[j]) would.
 * 1 <= m <= TID_MAX_MULTI.  The union of the patterns' bound columns is read
 * once.  Does not synchronise. */
int tid_match_multi(tid_ctx *ctx, const tid_store *st, const tid_pattern *pats, int m,
                    tid_set **outs);

/* Any number of patterns in two passes over the store per TID_BATCH_KEYS
 * distinct patterns: the multi-key search of Section 4.1 and of the
 * entailment steps of Section 5, grown to thousands of keys.  Every triple is
 * looked up, once per bound-position mask present, in a perfect-hash table of
 * the batch's keys held in shared memory, instead of being compared with
 * every key.  outs[j] receives the ascending index list of pats[j], exactly
 * as tid_match(pats[j]) would; equal patterns are scanned once and receive
 * views of one list; a pattern with no bound position goes through tid_match.
 * The union of the patterns' bound columns is read twice (a count pass sizes
 * every list, one synchronisation, a write pass fills them in order); the
 * lists of one sub-batch share one allocation, freed with the last of its
 * sets.  q >= 0; on error every outs[j] is NULL.  Errors: TID_ERR_ID if a
 * pattern value is negative.  Synchronises once per sub-batch. */
#define TID_BATCH_KEYS 1920
int tid_match_batch(tid_ctx *ctx, const tid_store *st, const tid_pattern *pats, int q,
                    tid_set **outs);

/* Testing aid for tid_match_batch (the paper has no counterpart): its host-side
 * planning of pats[0 .. q) -- the distinct (bound positions, key) pairs, split
 * into sub-batches of at most TID_BATCH_KEYS, each given a perfect-hash table
 * whose hash parameters are drawn from `seed`, seed + 1, ... (tid_match_batch
 * uses one fixed starting seed) and split in two when no seed gives a table --
 * followed by a check of every key the way the kernel looks it up: the
 * prefilter must admit it, and bucket, displacement and slot must lead to its
 * own entry, one key per slot.  No device work and no context.  *attempts
 * receives the number of table builds tried and *sub_batches the number of
 * sub-batches (either may be NULL).  Returns TID_OK; TID_ERR_ARG / TID_ERR_ID
 * for bad patterns; TID_ERR_CAPACITY if a check fails (a defect). */
int tid_batch_table_check(const tid_pattern *pats, int q, uint32_t seed, int *attempts, int *sub_batches);

/* What the autotuner of tid_match_batch chose for the last call on this
 * context that searched the store (the paper has no counterpart): the kernel
 * shape (TID_BATCH_DIRECT: every present mask looked up for every triple;
 * TID_BATCH_DIRECT_SKIP: the same, skipping masks no lane of a warp may answer;
 * TID_BATCH_QUEUE4 / TID_BATCH_QUEUE8: only the prefilter's candidates looked
 * up, 4 or 8 slots of 32 triples in flight), the keys per sub-batch and the
 * number of sub-batches; -1, 0, 0 before any such call.  Any pointer may be
 * NULL.  The choice is timed on the first call for each (GPU, store size, masks
 * read, log2 of the distinct keys) and kept for the process. */
#define TID_BATCH_DIRECT      0
#define TID_BATCH_DIRECT_SKIP 1
#define TID_BATCH_QUEUE4      2
#define TID_BATCH_QUEUE8      3
int tid_batch_tuning(const tid_ctx *ctx, int32_t *shape, int32_t *keys_per_sub_batch, int32_t *sub_batches);

/* A variant of tid_match that allocates nothing, for callers that may not
 * allocate device memory when they scan (for example a server that gave all
 * free device memory to its own pool at start-up, or a latency-critical loop
 * that cannot afford an allocation's implicit synchronisation).  The paper
 * has no counterpart; it is the same scan as tid_match.
 *
 * The caller passes the store columns s/p/o (n int32 each, device memory),
 * the output `out` (device memory, room for `cap` int32) and `count` (one
 * int64 in device memory), and the CUDA stream to run on (NULL = the legacy
 * default stream) of CUDA device `device`.  The call is stream-ordered and
 * does not wait: when the work completes, *count holds the number of matches
 * and out[0 .. min(count, cap)) the ascending matching positions (a count
 * above cap means the list was cut at cap).  *count is set to -1 when the
 * work starts and stays -1 if an in-kernel wait gave up.
 *
 * The scan's scratch (one status word per scan chunk, a ticket counter and an
 * error word) is a fixed array in device memory, TID_NOALLOC_MAX_CHUNKS status
 * words (32 KB), present on every GPU that loads the library until the
 * process exits.  The first call on a device looks up the array's device
 * address (with that device current); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents:
 * calls whose GPU work overlaps race on it, so order them (one stream, or
 * events).  Errors: TID_ERR_ARG (bad pointers, sizes or device, or another
 * device than this process's, as for tid_ctx_create), TID_ERR_ID
 * (negative pattern value), TID_ERR_CAPACITY (a GPU that would run more than
 * TID_NOALLOC_MAX_CHUNKS chunks per launch), TID_ERR_CUDA. */
#define TID_NOALLOC_MAX_CHUNKS 4096
int tid_match_noalloc(int device, void *cuda_stream, const int32_t *s, const int32_t *p,
                      const int32_t *o, int64_t n, tid_pattern pat, int32_t *out, int64_t cap,
                      int64_t *count);

/* ------------------------------------------------------------------------ */
/* operators on tuple sets -- Section 4                                      */
/* ------------------------------------------------------------------------ */

/* comparison of a FILTER predicate */
#define TID_CMP_EQ    0  /* x == a */
#define TID_CMP_NE    1  /* x != a */
#define TID_CMP_LT    2  /* x <  a */
#define TID_CMP_LE    3  /* x <= a */
#define TID_CMP_GT    4  /* x >  a */
#define TID_CMP_GE    5  /* x >= a */
#define TID_CMP_RANGE 6  /* a <= x <= b */

/* A FILTER predicate on variable `var`.  It compares the int32 ID itself:
 * literals encoded in ID order (an integer literal of value v has ID
 * 2^30 + v) make value ranges ID ranges (Section 4.3 proposes such an
 * order-preserving ID assignment).  An unbound value (0) never passes. */
typedef struct {
    int32_t var;
    int32_t op;
    int32_t a, b;
} tid_pred;

#define TID_MAX_PREDS 4

/* Result vector of one subquery (Section 4.2, vectors R_qi): for every index
 * in `idx` (a set from tid_match on the same store and pattern), the terms
 * at the pattern's variable slots.  Columns are the distinct variables of
 * pat.var[] in slot order (s, p, o).  A variable that occurs in two slots
 * keeps only triples whose two terms are equal.  The n_preds (<= 4)
 * predicates, all on variables of the pattern, are applied in the same pass
 * (Section 4.3: the filter is applied while the subquery's triples are
 * extracted).  The result is canonical: rows sorted lexicographically in
 * column order, without duplicates.  Synchronises once to size the output.
 * Errors: TID_ERR_ARG if the pattern has no variable, a bound slot carries a
 * variable, or a predicate names a variable not in the pattern. */
int tid_bind(tid_ctx *ctx, const tid_store *st, tid_pattern pat, const tid_set *idx,
             const tid_pred *preds, int n_preds, tid_set **out);

/* FILTER: rows of `in` for which every predicate holds, in the same order
 * (a canonical input gives a canonical output). */
int tid_filter(tid_ctx *ctx, const tid_set *in, const tid_pred *preds, int n_preds, tid_set **out);

#define TID_JOIN_AUTO       0
#define TID_JOIN_SORT_MERGE 1
#define TID_JOIN_HASH       2
/* or-ed into algo: a left outer join (SPARQL OPTIONAL; Section 4.2 names the
 * outer and left joins of the library the paper used).  Every row of L without
 * a match in R appears once, with R's other columns 0 (unbound).  Runs as a
 * sort-merge join (TID_JOIN_LEFT | TID_JOIN_HASH is TID_ERR_ARG). */
#define TID_JOIN_LEFT       0x100
/* or-ed into algo: a right outer join -- every row of R without a match in L
 * appears once, with L's other columns 0 -- and, with TID_JOIN_LEFT as well
 * (TID_JOIN_FULL), the full outer join.  Output columns as the inner join's
 * (L's, then R's others).  Built from the left join: right(L, R) is the left
 * join of R with L with its columns put in that order, full(L, R) the union of
 * left(L, R) and right(L, R).  Sort-merge only (with TID_JOIN_HASH:
 * TID_ERR_ARG). */
#define TID_JOIN_RIGHT      0x200
#define TID_JOIN_FULL       (TID_JOIN_LEFT | TID_JOIN_RIGHT)

/* Inner join of L and R on ALL their shared variables (Section 4.2 and its
 * relationship table: the shared term may come from any of S/P/O on either
 * side).  A pair joins when every shared column is equal and non-zero.
 * Output columns: L's, then R's non-shared ones in R's order (at most
 * TID_MAX_COLS).  No shared variable gives the cross product.  Algorithms:
 * sort-merge (sort both sides on the key, count matches per left row by
 * binary search, scan, write) or hash (group the smaller side by key in an
 * open-addressing table, probe with the other).  Output canonical.  The
 * count phase is followed by one synchronisation to size the output; more
 * than 2^31-1 output rows is TID_ERR_CAPACITY.  algo is TID_JOIN_AUTO,
 * TID_JOIN_SORT_MERGE or TID_JOIN_HASH, optionally or-ed with TID_JOIN_LEFT,
 * TID_JOIN_RIGHT or TID_JOIN_FULL for the outer joins above; anything else is
 * TID_ERR_ARG. */
int tid_join(tid_ctx *ctx, const tid_set *L, const tid_set *R, int algo, tid_set **out);

/* Set union of k >= 1 sets (Section 4.1).  The output schema lists the
 * variables of in[0], then the new ones of in[1], ...; a row from a branch
 * that lacks a variable carries 0 (unbound) there.  Duplicates are removed
 * (Section 4.3 keeps only distinct final values).  Output canonical. */
int tid_union(tid_ctx *ctx, const tid_set *const *in, int k, tid_set **out);

/* SELECT the n_vars listed variables (in that order) with DISTINCT
 * (Section 4.3).  Output canonical. */
int tid_project(tid_ctx *ctx, const tid_set *in, const int8_t *vars, int n_vars, tid_set **out);

/* A set from `rows` x `cols` int32 in host memory (row-major), labelled with
 * vars[0..cols-1] (distinct, 0..127); made canonical.  For inputs built
 * outside the library. */
int tid_set_from_host(tid_ctx *ctx, const int32_t *buf, int64_t rows, int cols,
                      const int8_t *vars, tid_set **out);

/* ------------------------------------------------------------------------ */
/* subquery plans -- Section 4.3, Fig. "Integration of several operations"   */
/* ------------------------------------------------------------------------ */

#define TID_OP_MATCH   1  /* search + extract one pattern (tid_match + tid_bind) */
#define TID_OP_FILTER  2  /* tid_filter(in[0], pred)                             */
#define TID_OP_JOIN    3  /* tid_join(in[0], in[1], algo)                        */
#define TID_OP_UNION   4  /* tid_union(in[0..n_in-1])                            */
#define TID_OP_PROJECT 5  /* tid_project(in[0], vars[0..n_vars-1])               */

typedef struct {
    int32_t op;
    int32_t n_in;       /* inputs used (JOIN 2, UNION 1..4, FILTER/PROJECT 1) */
    int32_t in[4];      /* indices of earlier nodes */
    tid_pattern pattern;/* MATCH */
    tid_pred pred;      /* FILTER */
    int32_t algo;       /* JOIN: TID_JOIN_* */
    int32_t n_vars;     /* PROJECT */
    int8_t vars[TID_MAX_COLS];
} tid_plan_node;

/* Evaluate a plan: nodes[i] may only read nodes[j], j < i; the last node is
 * the result.  All MATCH nodes are searched in one multi-pattern pass over
 * the store (up to TID_MAX_MULTI per pass); a FILTER whose input is a MATCH
 * read by nothing else is fused into that MATCH's extraction; joins run in
 * plan order (left-deep, as the paper's REL list).  The result is canonical
 * and equal to evaluating the nodes one by one with the calls above. */
int tid_exec(tid_ctx *ctx, const tid_store *st, const tid_plan_node *nodes, int n_nodes,
             tid_set **out);

/* The checks tid_exec and tid_server_submit make before anything runs: node
 * ops and input counts, inputs that are earlier nodes, join algorithm flags,
 * and every MATCH pattern (no negative ID, variables only on "?" slots, at
 * least one variable).  No device work and no context.  Returns TID_OK, or
 * TID_ERR_ARG / TID_ERR_ID as tid_exec would. */
int tid_plan_check(const tid_plan_node *nodes, int n_nodes);

/* ------------------------------------------------------------------------ */
/* tuple sets                                                                */
/* ------------------------------------------------------------------------ */

/* Number of rows (waits for the work that produces the set). */
int tid_set_rows(tid_set *set, int64_t *rows);

/* Shape of a set without waiting: column count, allocated row capacity,
 * variable ids (k entries), device column pointers (k entries, each valid for
 * `capacity` rows, of which the first `rows` are the set), and the device
 * address of the int64 row count.  Any output pointer may be NULL. */
int tid_set_info(const tid_set *set, int *cols, int64_t *capacity,
                 const int8_t **var_ids, int32_t *const **dev_cols,
                 const int64_t **dev_rows);

/* Copy a set to host memory, row-major (rows x cols int32).  If the set has
 * more than cap_rows rows nothing is copied, *rows_out receives the row count
 * and TID_ERR_CAPACITY is returned.  Synchronises. */
int tid_set_to_host(tid_set *set, int32_t *buf, int64_t cap_rows, int64_t *rows_out);

/* Free a set (NULL accepted).  Its memory is released stream-ordered on its
 * context's stream (work already queued there that reads it finishes first);
 * a set that views a shared allocation (tid_match_batch lists) releases it
 * with the last such set. */
int tid_set_free(tid_set *set);

/* ------------------------------------------------------------------------ */
/* RDFS entailment -- Section 5, Table "RDFS Entailment rules"               */
/* ------------------------------------------------------------------------ */

/* IDs of the vocabulary terms the rules name. */
typedef struct {
    int32_t type;             /* rdf:type */
    int32_t domain;           /* rdfs:domain */
    int32_t range;            /* rdfs:range */
    int32_t sub_property_of;  /* rdfs:subPropertyOf */
    int32_t sub_class_of;     /* rdfs:subClassOf */
} tid_rdfs_vocab;

/* the paper's step counts for one rule (its columns #Res1, #Dist1, #Res2,
 * #Dist2 and All): matches of the schema premise, its distinct join terms,
 * store triples found by the second search, their distinct join terms, and
 * distinct conclusions */
typedef struct {
    int64_t res1, dist1, res2, dist2, all;
} tid_entail_stats;

/* rules: 2 (s p o, p domain D => s type D), 3 (s p o, p range R => o type R),
 * 5 (p subPropertyOf q, q subPropertyOf r => p subPropertyOf r),
 * 7 (s p o, p subPropertyOf q => s q o), 9 (s type x, x subClassOf y =>
 * s type y), 11 (x subClassOf y, y subClassOf z => x subClassOf z) */
#define TID_RULE_R2  2
#define TID_RULE_R3  3
#define TID_RULE_R5  5
#define TID_RULE_R7  7
#define TID_RULE_R9  9
#define TID_RULE_R11 11

/* The conclusions of one rule over the store, as the paper evaluates it:
 * search the schema premise, take the distinct terms at its join position,
 * search the store for the triples of the other premise whose term at the join
 * position is one of them (one pass: a hash probe per triple), join the two
 * result vectors on that term, keep the distinct conclusions.  *out receives a
 * canonical three-column set (s, p, o) labelled 0, 1, 2; conclusions already in
 * the store are included.  stats may be NULL.  Errors: TID_ERR_ARG (unknown rule,
 * null vocab), TID_ERR_ID (a vocabulary ID <= 0).  Synchronises. */
int tid_entail(tid_ctx *ctx, const tid_store *st, int rule, const tid_rdfs_vocab *vocab,
               tid_set **out, tid_entail_stats *stats);

/* ------------------------------------------------------------------------ */
/* serving: a request loop over a resident store                             */
/* ------------------------------------------------------------------------ */
/*
 * The paper answers one query at a time (Section 4.3: split into subqueries,
 * search, extract, join).  A server keeps the store resident and answers a
 * stream of requests with continuous batching; the paper has no counterpart.
 *
 *  - Requests wait in one first-come-first-served queue.  A worker admits the
 *    requests at the head of the queue while their estimated device bytes fit
 *    in what is left of the budget (the head is always admitted when nothing
 *    else is admitted), up to max_wave of them: a wave.  Requests that arrive
 *    while a wave runs join the next wave of the first free worker.
 *  - Estimated bytes: a pattern's rows are estimated from value counts of a
 *    strided sample of the store (the least frequent bound value wins); a
 *    plan's bytes are the sum over its nodes of estimated rows x 4 bytes x
 *    (columns + 1), joins estimated as their larger input, unions as the sum.
 *  - With batch_scans = 1, every MATCH node of every request of a wave is
 *    searched by one tid_match_batch call; each request then runs the rest of
 *    its plan.  With batch_scans = 0 each request searches alone (tid_match
 *    for an index request, tid_exec for a plan): with max_wave = 1 and one
 *    worker this is one launch per query, the server's own baseline.
 *  - Workers run on their own contexts and streams, so one wave's operators
 *    overlap the next wave's scan on the GPU.
 *  - A request's result is copied to host memory owned by the server until
 *    tid_server_release.  Its latency runs from its arrival time (given at
 *    submission on the tid_server_now_ns clock, or the submission time) to the
 *    moment its result is in host memory.
 *  - A result does not depend on what else is in the wave: every path returns
 *    the canonical set (index lists: the ascending list).
 */
typedef struct tid_server tid_server;

typedef struct {
    int32_t workers;       /* worker threads, each with its own context and stream (1..16) */
    int32_t max_wave;      /* requests per wave (>= 1) */
    int32_t batch_scans;   /* 1: a wave shares one batched search; 0: each request searches alone */
    int32_t reserved;      /* set to 0 */
    int64_t budget_bytes;  /* estimated device bytes of admitted requests; 0 = unlimited */
} tid_server_config;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t waves;               /* waves run */
    int64_t max_wave_seen;       /* largest wave */
    int64_t peak_admitted_bytes; /* largest sum of estimates admitted at once */
    int64_t scan_patterns;       /* MATCH nodes searched */
    int64_t budget_waits;        /* requests that reached the queue's head and waited for budget */
} tid_server_stats;

#define TID_REQ_INDEX 1  /* nodes = one MATCH node; result: its ascending index list (one column, -1) */
#define TID_REQ_PLAN  2  /* result: the plan's canonical tuple set (as tid_exec)                      */

/* Server on CUDA device `device` over the store s/p/o (n int32 each, device
 * memory, borrowed: unchanged and valid until tid_server_destroy).  Waits for
 * the device once (work still writing the columns on any stream finishes),
 * reads a strided sample of every column for its estimates, and starts the
 * workers.  Errors: TID_ERR_ARG (bad configuration), TID_ERR_OOM,
 * TID_ERR_CUDA. */
int tid_server_create(int device, const int32_t *s, const int32_t *p, const int32_t *o, int64_t n,
                      const tid_server_config *cfg, tid_server **out);

/* Nanoseconds on the server clock (steady, process-wide). */
int64_t tid_server_now_ns(void);

/* Queue a request (nodes are copied); *id receives its id.  arrival_ns <= 0
 * means now.  The plan is checked here: TID_ERR_ARG / TID_ERR_ID as tid_exec. */
int tid_server_submit(tid_server *srv, int kind, const tid_plan_node *nodes, int n_nodes, int64_t arrival_ns,
                      int64_t *id);

/* Wait up to timeout_ms (< 0: forever) for request id: TID_OK once it has
 * finished (successfully or not), TID_ERR_TIMEOUT if it has not yet. */
int tid_server_wait(tid_server *srv, int64_t id, int64_t timeout_ms);

/* A finished request: its status (TID_OK or the error of its evaluation),
 * columns, variable ids (up to TID_MAX_COLS), rows, host data (rows x cols
 * int32, row-major; owned by the server until tid_server_release) and latency.
 * Any output pointer may be NULL.  TID_ERR_ARG if id is unknown or unfinished. */
int tid_server_result(tid_server *srv, int64_t id, int *status, int *cols, int8_t *vars, int64_t *rows,
                      const int32_t **data, int64_t *latency_ns);

/* Forget a finished request and its host data (the data pointer returned by
 * tid_server_result is invalid afterwards).  Any thread may call any
 * tid_server_* function; a release while another thread waits on the same id
 * is safe (that wait returns TID_OK, the request having finished). */
int tid_server_release(tid_server *srv, int64_t id);

/* Counters since tid_server_create (see tid_server_stats). */
int tid_server_get_stats(tid_server *srv, tid_server_stats *out);

/* Finish every queued request, stop the workers and free the server. */
int tid_server_destroy(tid_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* TID_H_ */
