/*
 * Trivial errors of a detector error model: every set S of at most w columns
 * with H 1_S = 0 and O 1_S = 0 over GF(2) (App. D: the rows of the detector
 * degeneracy matrix beyond the stabilizers).  Input construction only; no
 * decoder arithmetic.
 *
 * Depth-first search over connected supports.  S starts with its smallest
 * column c1; while some detector is unsatisfied, the next column must flip
 * the lowest such detector d (any trivial superset has to cancel d), so the
 * search branches over the columns of detector d greater than c1 and not yet
 * in S.  Every trivial error whose support is connected through shared
 * detectors is reached; for the BB detector models with w <= 5 every trivial
 * error is connected (no trivial error of weight <= 2 exists, so a
 * disconnected one has weight >= 6).  A set may be reached along several
 * orders; the caller removes repeats.  Pruning: a column flips at most cmax
 * detectors, so more than cmax * (w - |S|) unsatisfied detectors cannot be
 * cleared.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int M, N, K, w, cmax;
    const int32_t *row_ptr, *row_col;   /* detectors -> columns (CSR) */
    const int32_t *col_ptr, *col_row;   /* columns -> detectors (CSC) */
    const uint64_t *obs;                /* column -> observable bits (K <= 64) */
    uint8_t *par;                       /* detector parities of S */
    int32_t *unsat;                     /* unsatisfied detectors, unsorted */
    int n_unsat;
    int32_t stack[8];
    uint8_t *in_set;
    int32_t *out;                       /* found sets, w entries each (-1 padded) */
    int64_t n_out, cap_out;
    int overflow;
} search;

static void flip(search *s, int c)
{
    for (int a = s->col_ptr[c]; a < s->col_ptr[c + 1]; ++a) {
        const int d = s->col_row[a];
        s->par[d] ^= 1;
        if (s->par[d]) {
            s->unsat[s->n_unsat++] = d;
        } else {
            for (int k = 0; k < s->n_unsat; ++k)
                if (s->unsat[k] == d) { s->unsat[k] = s->unsat[--s->n_unsat]; break; }
        }
    }
}

static void emit(search *s, int depth)
{
    if (s->n_out >= s->cap_out) { s->overflow = 1; return; }
    int32_t *o = s->out + s->n_out * s->w;
    for (int k = 0; k < s->w; ++k) o[k] = k < depth ? s->stack[k] : -1;
    s->n_out++;
}

static void dfs(search *s, int depth, uint64_t obs)
{
    if (s->overflow) return;
    if (s->n_unsat == 0) {
        if (obs == 0) emit(s, depth);
        return;
    }
    if (depth == s->w || s->n_unsat > s->cmax * (s->w - depth)) return;
    int d = s->unsat[0];
    for (int k = 1; k < s->n_unsat; ++k)
        if (s->unsat[k] < d) d = s->unsat[k];
    const int c1 = s->stack[0];
    for (int a = s->row_ptr[d]; a < s->row_ptr[d + 1]; ++a) {
        const int c = s->row_col[a];
        if (c <= c1 || s->in_set[c]) continue;
        s->stack[depth] = c;
        s->in_set[c] = 1;
        flip(s, c);
        dfs(s, depth + 1, obs ^ s->obs[c]);
        flip(s, c);
        s->in_set[c] = 0;
    }
}

/* Returns the number of sets written to out (each w columns, -1 padded),
 * or -1 if cap_out sets were not enough. */
int64_t trivial_errors(int M, int N, int K, int w, const int32_t *row_ptr, const int32_t *row_col,
                       const int32_t *col_ptr, const int32_t *col_row, const uint64_t *obs, int32_t *out,
                       int64_t cap_out)
{
    if (w < 1 || w > 8 || K > 64) return -1;
    search s;
    memset(&s, 0, sizeof(s));
    s.M = M; s.N = N; s.K = K; s.w = w;
    s.row_ptr = row_ptr; s.row_col = row_col; s.col_ptr = col_ptr; s.col_row = col_row; s.obs = obs;
    for (int c = 0; c < N; ++c)
        if (col_ptr[c + 1] - col_ptr[c] > s.cmax) s.cmax = col_ptr[c + 1] - col_ptr[c];
    s.par = (uint8_t *)calloc((size_t)M, 1);
    s.unsat = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s.cmax * w + 1));
    s.in_set = (uint8_t *)calloc((size_t)N, 1);
    s.out = out;
    s.cap_out = cap_out;
    for (int c1 = 0; c1 < N && !s.overflow; ++c1) {
        s.stack[0] = c1;
        s.in_set[c1] = 1;
        flip(&s, c1);
        dfs(&s, 1, obs[c1]);
        flip(&s, c1);
        s.in_set[c1] = 0;
    }
    free(s.par);
    free(s.unsat);
    free(s.in_set);
    return s.overflow ? -1 : s.n_out;
}
