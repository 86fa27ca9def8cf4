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
 * context creates and owns.  On success *out receives the context. */
int tid_ctx_create(int device, void *cuda_stream, tid_ctx **out);

/* Wait for all work on the context's stream; returns TID_ERR_TIMEOUT if an
 * in-kernel wait gave up since the last check, TID_ERR_CUDA on a CUDA error. */
int tid_ctx_sync(tid_ctx *ctx);

/* Destroy the context (synchronises first).  NULL is accepted. */
int tid_ctx_destroy(tid_ctx *ctx);

/* Message of the last failing call on this thread ("" if none). */
const char *tid_last_error(void);

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
 * for the tuple-set calls to return sets.  Returns after the copies are
 * queued on the context stream. */
int tid_load(tid_ctx *ctx, const int32_t *s, const int32_t *p, const int32_t *o,
             int64_t n, int where, int copy, tid_store **out);

/* Number of triples and the device columns of a store. */
int tid_store_info(const tid_store *st, int64_t *n, const int32_t **s,
                   const int32_t **p, const int32_t **o);

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

int tid_set_free(tid_set *set);

#ifdef __cplusplus
}
#endif

#endif /* TID_H_ */
