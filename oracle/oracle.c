/*
 * TripleID-Q CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, single-threaded, obviously-correct C for what the query hot path
 * computes.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the product library never links or calls it, and
 * it includes no header and shares no code with the CUDA sources.
 *
 * Conventions (Section 3 of the paper): a triple is (S[i], P[i], O[i]) with
 * 32-bit IDs; the key value 0 stands for the free variable "?".  Tuple sets
 * here are ROW-MAJOR int32 arrays (n rows x k columns).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Single pattern search.  Section 3, Algorithm 1 ("Parallel Search for     */
/* TripleID"): a triple answers the key when every key component is either  */
/* 0 ("?") or equal to the triple's component.  The positions found are     */
/* listed in ascending order (positionArray marks triple positions).        */
/* out may be NULL (count only).  Returns the number of matches.           */
/* ------------------------------------------------------------------------ */
static int triple_matches(int32_t s, int32_t p, int32_t o,
                          int32_t ks, int32_t kp, int32_t ko)
{
    if (ks != 0 && s != ks) return 0;
    if (kp != 0 && p != kp) return 0;
    if (ko != 0 && o != ko) return 0;
    return 1;
}

int64_t or_match(const int32_t *S, const int32_t *P, const int32_t *O, int64_t n,
                 int32_t ks, int32_t kp, int32_t ko, int32_t *out)
{
    int64_t h = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (triple_matches(S[i], P[i], O[i], ks, kp, ko)) {
            if (out) out[h] = (int32_t)i;
            ++h;
        }
    }
    return h;
}

/* ------------------------------------------------------------------------ */
/* Several keys in one pass.  Section 4.1 (union operation): the key array  */
/* holds m keys (3 IDs each); every triple is marked with the list of the   */
/* subqueries it answers (positionArray[i].query), and one triple may       */
/* answer several.  Here the marks are emitted as one ascending position    */
/* list per subquery.  counts[j] receives the size of list j; outs may be   */
/* NULL (count only), else outs[j] must hold counts[j] entries.             */
/* ------------------------------------------------------------------------ */
void or_match_multi(const int32_t *S, const int32_t *P, const int32_t *O, int64_t n,
                    const int32_t *keys, int m, int64_t *counts, int32_t **outs)
{
    for (int j = 0; j < m; ++j) counts[j] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int j = 0; j < m; ++j) {
            if (triple_matches(S[i], P[i], O[i], keys[3 * j], keys[3 * j + 1], keys[3 * j + 2])) {
                if (outs) outs[j][counts[j]] = (int32_t)i;
                counts[j]++;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Result vector of one subquery (Section 4.2, vectors R_qi): for each      */
/* found triple, the terms at its variable positions.  var[j] is the        */
/* variable id at slot j (s, p, o) or -1; out_vars[c] (c < k) is the        */
/* variable of output column c.  A variable that occurs at two slots must   */
/* take the same value at both, else the triple yields no row.  Returns the */
/* number of rows written to out (row-major, k columns).                    */
/* ------------------------------------------------------------------------ */
int64_t or_bind(const int32_t *S, const int32_t *P, const int32_t *O,
                const int32_t *idx, int64_t h, const int8_t *var,
                int k, const int8_t *out_vars, int32_t *out)
{
    int64_t r = 0;
    for (int64_t t = 0; t < h; ++t) {
        int64_t i = idx[t];
        int32_t term[3] = {S[i], P[i], O[i]};
        int ok = 1;
        int32_t row[8];
        for (int c = 0; c < k && ok; ++c) {
            int have = 0;
            for (int j = 0; j < 3; ++j) {
                if (var[j] != out_vars[c]) continue;
                if (!have) { row[c] = term[j]; have = 1; }
                else if (row[c] != term[j]) ok = 0;
            }
        }
        if (!ok) continue;
        memcpy(out + r * k, row, (size_t)k * sizeof(int32_t));
        ++r;
    }
    return r;
}

/* ------------------------------------------------------------------------ */
/* Row order.  Lexicographic by a list of columns, as signed int32.         */
/* A stable bottom-up merge sort of a row permutation.                      */
/* ------------------------------------------------------------------------ */
static int row_cmp(const int32_t *a, const int32_t *b, const int *cols, int nc)
{
    for (int c = 0; c < nc; ++c) {
        int32_t x = a[cols[c]], y = b[cols[c]];
        if (x < y) return -1;
        if (x > y) return 1;
    }
    return 0;
}

static int sort_perm(const int32_t *rows, int k, int64_t n,
                     const int *cols, int nc, int64_t *perm)
{
    int64_t *tmp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!tmp) return -1;
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t w = 1; w < n; w *= 2) {
        for (int64_t lo = 0; lo < n; lo += 2 * w) {
            int64_t mid = lo + w < n ? lo + w : n;
            int64_t hi = lo + 2 * w < n ? lo + 2 * w : n;
            int64_t a = lo, b = mid, o = lo;
            while (a < mid && b < hi) {
                /* take from the left run on ties: stable */
                if (row_cmp(rows + perm[b] * k, rows + perm[a] * k, cols, nc) < 0)
                    tmp[o++] = perm[b++];
                else
                    tmp[o++] = perm[a++];
            }
            while (a < mid) tmp[o++] = perm[a++];
            while (b < hi) tmp[o++] = perm[b++];
        }
        memcpy(perm, tmp, (size_t)n * sizeof(int64_t));
    }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Canonical form of a tuple set: rows sorted lexicographically in column   */
/* order, duplicates removed (the final results keep only distinct values,  */
/* Section 4.3).  In place; returns the new row count, or -1 on OOM.        */
/* ------------------------------------------------------------------------ */
int64_t or_canonical(int32_t *rows, int64_t n, int k)
{
    if (n <= 0 || k <= 0) return n;
    int cols[8];
    for (int c = 0; c < k; ++c) cols[c] = c;
    int64_t *perm = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int32_t *tmp = (int32_t *)malloc((size_t)n * (size_t)k * sizeof(int32_t));
    if (!perm || !tmp || sort_perm(rows, k, n, cols, k, perm) != 0) {
        free(perm); free(tmp); return -1;
    }
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *r = rows + perm[i] * k;
        if (m > 0 && row_cmp(tmp + (m - 1) * k, r, cols, k) == 0) continue;
        memcpy(tmp + m * k, r, (size_t)k * sizeof(int32_t));
        ++m;
    }
    memcpy(rows, tmp, (size_t)m * (size_t)k * sizeof(int32_t));
    free(perm); free(tmp);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Join of two result vectors on their shared variables (Section 4.2,       */
/* Table "Relationship between two triple patterns": the shared term may    */
/* sit at any of S/P/O on either side).  A pair (l, r) joins when every     */
/* key column pair is equal; the value 0 (an unbound variable) never        */
/* equals anything.  The output row is L's row followed by R's rest         */
/* columns.  Plain nested loop over L x R.  out may be NULL (count only).   */
/* ------------------------------------------------------------------------ */
static int keys_join(const int32_t *l, const int32_t *r, int nk,
                     const int *lkey, const int *rkey)
{
    for (int c = 0; c < nk; ++c) {
        int32_t x = l[lkey[c]];
        if (x == 0 || x != r[rkey[c]]) return 0;
    }
    return 1;
}

int64_t or_join_nested(const int32_t *L, int64_t nl, int kl,
                       const int32_t *R, int64_t nr, int kr,
                       int nk, const int *lkey, const int *rkey,
                       int nrest, const int *rrest, int32_t *out)
{
    int64_t m = 0;
    int ko = kl + nrest;
    for (int64_t i = 0; i < nl; ++i) {
        const int32_t *l = L + i * kl;
        for (int64_t j = 0; j < nr; ++j) {
            const int32_t *r = R + j * kr;
            if (!keys_join(l, r, nk, lkey, rkey)) continue;
            if (out) {
                int32_t *o = out + m * ko;
                memcpy(o, l, (size_t)kl * sizeof(int32_t));
                for (int c = 0; c < nrest; ++c) o[kl + c] = r[rrest[c]];
            }
            ++m;
        }
    }
    return m;
}

/* ------------------------------------------------------------------------ */
/* The same join by sorting both sides on the key columns and merging equal */
/* key groups (the sort-then-merge-join route of Section 4.2/4.3).  Used    */
/* only where L x R is too large for the nested loop; it is checked against */
/* or_join_nested on every case where both run.  Returns -1 on OOM.         */
/* ------------------------------------------------------------------------ */
static int has_zero_key(const int32_t *row, int nk, const int *key)
{
    for (int c = 0; c < nk; ++c) if (row[key[c]] == 0) return 1;
    return 0;
}

static int key_cmp(const int32_t *l, const int *lkey, const int32_t *r, const int *rkey, int nk)
{
    for (int c = 0; c < nk; ++c) {
        int32_t x = l[lkey[c]], y = r[rkey[c]];
        if (x < y) return -1;
        if (x > y) return 1;
    }
    return 0;
}

int64_t or_join_sortmerge(const int32_t *L, int64_t nl, int kl,
                          const int32_t *R, int64_t nr, int kr,
                          int nk, const int *lkey, const int *rkey,
                          int nrest, const int *rrest, int32_t *out)
{
    int64_t *pl = (int64_t *)malloc((size_t)(nl > 0 ? nl : 1) * sizeof(int64_t));
    int64_t *pr = (int64_t *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    if (!pl || !pr || sort_perm(L, kl, nl, lkey, nk, pl) || sort_perm(R, kr, nr, rkey, nk, pr)) {
        free(pl); free(pr); return -1;
    }
    int64_t m = 0, a = 0, b = 0;
    int ko = kl + nrest;
    while (a < nl && b < nr) {
        const int32_t *l = L + pl[a] * kl;
        const int32_t *r = R + pr[b] * kr;
        if (has_zero_key(l, nk, lkey)) { ++a; continue; }
        if (has_zero_key(r, nk, rkey)) { ++b; continue; }
        int c = key_cmp(l, lkey, r, rkey, nk);
        if (c < 0) { ++a; continue; }
        if (c > 0) { ++b; continue; }
        /* equal key: the groups [a, a2) x [b, b2) all join */
        int64_t a2 = a + 1, b2 = b + 1;
        while (a2 < nl && key_cmp(L + pl[a2] * kl, lkey, r, rkey, nk) == 0) ++a2;
        while (b2 < nr && key_cmp(l, lkey, R + pr[b2] * kr, rkey, nk) == 0) ++b2;
        for (int64_t x = a; x < a2; ++x) {
            for (int64_t y = b; y < b2; ++y) {
                if (out) {
                    int32_t *o = out + m * ko;
                    memcpy(o, L + pl[x] * kl, (size_t)kl * sizeof(int32_t));
                    const int32_t *rr = R + pr[y] * kr;
                    for (int q = 0; q < nrest; ++q) o[kl + q] = rr[rrest[q]];
                }
                ++m;
            }
        }
        a = a2; b = b2;
    }
    free(pl); free(pr);
    return m;
}

/* ------------------------------------------------------------------------ */
/* FILTER on one column (Section 4.3 filters found values; on integer IDs   */
/* the comparison runs on the order-preserving encoding).  A row whose      */
/* column is 0 (unbound) never passes.  Keeps row order.                    */
/*   op: 0 EQ, 1 NE, 2 LT, 3 LE, 4 GT, 5 GE, 6 RANGE (a <= x <= b)          */
/* ------------------------------------------------------------------------ */
int64_t or_filter(const int32_t *rows, int64_t n, int k, int col,
                  int op, int32_t a, int32_t b, int32_t *out)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t x = rows[i * k + col];
        int keep;
        if (x == 0) keep = 0;
        else switch (op) {
            case 0: keep = x == a; break;
            case 1: keep = x != a; break;
            case 2: keep = x < a; break;
            case 3: keep = x <= a; break;
            case 4: keep = x > a; break;
            case 5: keep = x >= a; break;
            case 6: keep = a <= x && x <= b; break;
            default: keep = 0;
        }
        if (keep) {
            memcpy(out + m * k, rows + i * k, (size_t)k * sizeof(int32_t));
            ++m;
        }
    }
    return m;
}
