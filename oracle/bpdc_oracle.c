/*
 * bpdc_oracle.c -- plain FP64 CPU reference of BP+DC decoding
 * (Tsubouchi, Yamasaki, Tamiya, "Degeneracy Cutting: A Local and Efficient
 * Post-Processing for Belief Propagation Decoding of qLDPC Codes",
 * arXiv 2510.08695).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or helper with the CUDA decoder; it is written for reading against
 * the paper, not for speed:
 *
 *   - Sec. II.C.1: flooding BP.  Every iteration first sends a message from
 *     every variable node to each of its checks, then a message from every
 *     check back to each of its variables; afterwards the posteriors are
 *     updated, a hard decision is made (Eq. 4) and the run stops as soon as
 *     the hard decision reproduces the syndrome, else after T_iter
 *     iterations.
 *   - Check rules (Sec. II.C.1 cites them): normalized min-sum and
 *     product-sum, written per edge from their definitions, O(d^2) per check;
 *     the product-sum value 2 atanh(prod tanh(q/2)) is folded over the other
 *     edges with the pairwise rule a [+] b = 2 atanh(tanh(a/2) tanh(b/2)) in
 *     its log form min(a,b) + log(1 + e^-(a+b)) - log(1 + e^-|a-b|), which
 *     stays exact at every magnitude up to the cap (tanh(q/2) rounds to 1
 *     above |q| ~ 37 in FP64, and -log tanh(q/2) underflows above ~709).
 *   - Algorithm 1: run BP; if it fails, for every row of the degeneracy
 *     matrix D pick the support variable of lowest posterior error
 *     probability (= highest posterior LLR), take the union of the picks,
 *     delete those columns (DeleteColumns / DeleteEntries), run BP again and
 *     pad the cut coordinates with zeros (PadWithZeros).
 *   - Algorithm 2: the same cut applied by setting the cut priors to 0
 *     (LLR = +infinity) instead of deleting columns.
 *
 * Readings of points the paper leaves open (each one is a parameter or a
 * documented constant here):
 *   - min-sum scale alpha is a parameter (the workloads use 0.625);
 *   - sgn(0) = +1 in the sign product;
 *   - a check-to-variable magnitude is capped at ORACLE_LLR_CAP (1e30): the
 *     minimum over an empty set (a check whose other neighbours were all
 *     cut) is the cap, and so are messages that would otherwise grow without
 *     bound over very long runs;
 *   - hard decision e_j = 1 iff posterior LLR <= 0 (p_hat >= 1/2, Eq. 4);
 *   - the convergence test runs before the first iteration (on the priors)
 *     and after every iteration;
 *   - ties in the cut selection ("selected at random", Sec. III.A) are
 *     broken by a window plus a keyed hash: the candidates of a row are the
 *     support variables with L_j >= L_max - tie_rel * max(1, |L_max|); the
 *     candidate of rank h(tie_seed, shot * rows(D) + row) mod |candidates|
 *     in ascending column order is cut, h being the SplitMix64 output
 *     function (Steele, Lea & Flood 2014);
 *   - second BP priors: the original priors p (the paper's choice for BB
 *     codes, Sec. III.B) or, with dc_prior = 1, the first-run posterior
 *     p_hat clamped to [1e-12, 1/2] (Algorithm 1 as printed);
 *   - cut variables report e_j = 0 and posterior LLR = +infinity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_LLR_CAP 1e30

typedef struct {
    int32_t M, N;                       /* H is M x N */
    const int32_t *h_row_ptr, *h_col;   /* H in CSR */
    int32_t Md;                         /* D is Md x N */
    const int32_t *d_row_ptr, *d_col;   /* D in CSR, ascending columns per row */
    int32_t K;                          /* L is K x N */
    const int32_t *l_row_ptr, *l_col;   /* L in CSR */
    const double *prior;                /* p_j */
} oracle_problem;

typedef struct {
    int32_t variant;    /* 0: normalized min-sum, 1: product-sum */
    double alpha;       /* min-sum scale factor */
    int32_t max_iter;   /* T_iter */
    int32_t dc_enable;  /* run degeneracy cutting when BP fails */
    int32_t dc_prior;   /* 0: second BP on priors p; 1: on the first-run posterior */
    int32_t cut_form;   /* 0: DeleteColumns (Algorithm 1); 1: zero prior (Algorithm 2) */
    double tie_rel;     /* tie window for the cut selection */
    uint64_t tie_seed;  /* key of the tie-break hash */
} oracle_opts;

/* SplitMix64 output number ctr of the stream whose state starts at key. */
uint64_t oracle_hash(uint64_t key, uint64_t ctr)
{
    uint64_t z = key + (ctr + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* A Tanner graph with both adjacency orders: row lists (check -> edges) and
 * column lists (variable -> edges).  Edge e is the e-th nonzero of H in CSR
 * order; it joins check edge_row[e] and variable edge_col[e]. */
typedef struct {
    int M, N, E;
    const int32_t *row_ptr, *col;   /* CSR: edges of check i are row_ptr[i]..row_ptr[i+1]-1 */
    int32_t *edge_row;              /* check of each edge */
    int32_t *col_ptr, *col_edges;   /* variable j owns edges col_edges[col_ptr[j]..col_ptr[j+1]-1] */
} tanner;

static void tanner_build(tanner *g, int M, int N, const int32_t *row_ptr, const int32_t *col)
{
    int E = row_ptr[M];
    g->M = M; g->N = N; g->E = E;
    g->row_ptr = row_ptr; g->col = col;
    g->edge_row = (int32_t *)malloc(sizeof(int32_t) * (E > 0 ? E : 1));
    g->col_ptr = (int32_t *)calloc((size_t)N + 1, sizeof(int32_t));
    g->col_edges = (int32_t *)malloc(sizeof(int32_t) * (E > 0 ? E : 1));
    for (int i = 0; i < M; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            g->edge_row[e] = i;
            g->col_ptr[col[e] + 1]++;
        }
    for (int j = 0; j < N; ++j) g->col_ptr[j + 1] += g->col_ptr[j];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * ((size_t)N + 1));
    memcpy(fill, g->col_ptr, sizeof(int32_t) * ((size_t)N + 1));
    for (int e = 0; e < E; ++e) g->col_edges[fill[col[e]]++] = e;
    free(fill);
}

static void tanner_free(tanner *g)
{
    free(g->edge_row); free(g->col_ptr); free(g->col_edges);
}

static double sgn(double x) { return x < 0.0 ? -1.0 : 1.0; }

/* Magnitude of the product-sum of two messages of magnitudes a, b >= 0:
 * 2 atanh(tanh(a/2) tanh(b/2)) = log((1 + e^-(a+b)) / (e^-a + e^-b)), which
 * rearranges to min(a,b) + log(1 + e^-(a+b)) - log(1 + e^-|a-b|).  +inf is
 * the identity (a cut or absent neighbour), and the result lies in
 * [0, min(a,b)]. */
static double boxplus(double a, double b)
{
    double d = (a == b) ? 0.0 : fabs(a - b);
    double r = fmin(a, b) + log1p(exp(-(a + b))) - log1p(exp(-d));
    return r > 0.0 ? r : 0.0;
}

/* Check-to-variable message on edge e of check i: the check tells its
 * variable what the parity constraint s_i implies given the messages arriving
 * on all of its *other* edges. */
static double check_message(const tanner *g, int i, int e, int s_i, const double *q,
                            int variant, double alpha)
{
    double syn_sign = s_i ? -1.0 : 1.0;
    if (variant == 0) {
        /* normalized min-sum: alpha * (-1)^s_i * prod sgn(q) * min |q| */
        double sign = syn_sign, mag = INFINITY;
        for (int f = g->row_ptr[i]; f < g->row_ptr[i + 1]; ++f) {
            if (f == e) continue;
            sign *= sgn(q[f]);
            if (fabs(q[f]) < mag) mag = fabs(q[f]);
        }
        if (mag > ORACLE_LLR_CAP) mag = ORACLE_LLR_CAP;
        return alpha * sign * mag;
    } else {
        /* product-sum: (-1)^s_i * sign * 2 atanh( prod |tanh(q / 2)| ), the
         * product taken pairwise with boxplus (the empty product is +inf) */
        double sign = syn_sign, mag = INFINITY;
        for (int f = g->row_ptr[i]; f < g->row_ptr[i + 1]; ++f) {
            if (f == e) continue;
            sign *= sgn(q[f]);
            mag = boxplus(mag, fabs(q[f]));
        }
        if (!(mag < ORACLE_LLR_CAP)) mag = ORACLE_LLR_CAP;
        return sign * mag;
    }
}

static int syndrome_matches(const tanner *g, const uint8_t *e_hat, const uint8_t *s)
{
    for (int i = 0; i < g->M; ++i) {
        int par = 0;
        for (int f = g->row_ptr[i]; f < g->row_ptr[i + 1]; ++f) par ^= e_hat[g->col[f]];
        if (par != (s[i] & 1)) return 0;
    }
    return 1;
}

/* BP_decode(H, s, lambda, T) of Algorithm 1 on graph g.
 * lam: prior LLRs ln((1-p)/p); +INFINITY marks a variable with prior 0.
 * Writes the hard decision and posterior LLRs; returns 1 if the hard decision
 * reproduces s.  With early_stop = 0 all T iterations run (used to compare
 * against exact marginals on trees). */
static int bp_run(const tanner *g, const uint8_t *s, const double *lam, int T, int variant,
                  double alpha, int early_stop, uint8_t *e_hat, double *post, int *iters,
                  double *q, double *r)
{
    const int M = g->M, N = g->N, E = g->E;
    /* iteration 0: every variable announces its prior */
    for (int e = 0; e < E; ++e) q[e] = lam[g->col[e]];
    for (int j = 0; j < N; ++j) { post[j] = lam[j]; e_hat[j] = post[j] <= 0.0; }
    int ok = syndrome_matches(g, e_hat, s);
    if (ok && early_stop) { *iters = 0; return 1; }
    for (int t = 1; t <= T; ++t) {
        /* checks -> variables */
        for (int i = 0; i < M; ++i)
            for (int e = g->row_ptr[i]; e < g->row_ptr[i + 1]; ++e)
                r[e] = check_message(g, i, e, s[i] & 1, q, variant, alpha);
        /* variables: posterior and the next variable -> check messages */
        for (int j = 0; j < N; ++j) {
            double sum = lam[j];
            for (int a = g->col_ptr[j]; a < g->col_ptr[j + 1]; ++a) sum += r[g->col_edges[a]];
            post[j] = sum;
            for (int a = g->col_ptr[j]; a < g->col_ptr[j + 1]; ++a) {
                int e = g->col_edges[a];
                double ext = lam[j];
                for (int b = g->col_ptr[j]; b < g->col_ptr[j + 1]; ++b)
                    if (b != a) ext += r[g->col_edges[b]];
                q[e] = ext;
            }
            e_hat[j] = post[j] <= 0.0;   /* Eq. 4 */
        }
        ok = syndrome_matches(g, e_hat, s);
        if (ok && early_stop) { *iters = t; return 1; }
    }
    *iters = T;
    return ok;
}

static double prior_llr(double p)
{
    return log((1.0 - p) / p);   /* p = 0 gives +infinity */
}

int oracle_bp(const oracle_problem *P, const oracle_opts *o, const uint8_t *s, const double *lam,
              int early_stop, uint8_t *e_hat, double *post, int32_t *iters)
{
    tanner g;
    tanner_build(&g, P->M, P->N, P->h_row_ptr, P->h_col);
    double *q = (double *)malloc(sizeof(double) * (g.E > 0 ? g.E : 1));
    double *r = (double *)malloc(sizeof(double) * (g.E > 0 ? g.E : 1));
    int it = 0;
    int ok = bp_run(&g, s, lam, o->max_iter, o->variant, o->alpha, early_stop, e_hat, post, &it, q, r);
    *iters = it;
    free(q); free(r);
    tanner_free(&g);
    return ok;
}

/* The selection step of Algorithm 1: for every row h of D pick argmin_{i in supp h}
 * p_hat_i (= argmax of the posterior LLR) and add it to the cut set.  The
 * union makes the result independent of the row order. */
void oracle_dc_select(const oracle_problem *P, const oracle_opts *o, const double *post,
                      uint64_t shot, uint8_t *cut)
{
    memset(cut, 0, (size_t)P->N);
    int32_t cand[4096];
    for (int row = 0; row < P->Md; ++row) {
        int b = P->d_row_ptr[row], end = P->d_row_ptr[row + 1];
        if (b == end) continue;
        double lmax = -INFINITY;
        for (int a = b; a < end; ++a)
            if (post[P->d_col[a]] > lmax) lmax = post[P->d_col[a]];
        double thr = isfinite(lmax) ? lmax - o->tie_rel * fmax(1.0, fabs(lmax)) : lmax;
        int nc = 0;
        for (int a = b; a < end && nc < 4096; ++a)
            if (post[P->d_col[a]] >= thr) cand[nc++] = P->d_col[a];
        uint64_t h = oracle_hash(o->tie_seed, shot * (uint64_t)P->Md + (uint64_t)row);
        cut[cand[h % (uint64_t)nc]] = 1;
    }
}

/* Algorithm 1 for one shot.  Returns status: 0 BP converged, 1 BP+DC
 * converged, 2 failure (Sec. III.A: no repetition of the cut). */
static int decode_shot(const oracle_problem *P, const oracle_opts *o, const tanner *g,
                       const double *lam, const uint8_t *s, uint64_t shot,
                       uint8_t *e_hat, double *post, double *post1, uint8_t *cut,
                       int32_t *it1, int32_t *it2, double *q, double *r,
                       double *lam2, int32_t *keep, int32_t *sub_row_ptr, int32_t *sub_col,
                       uint8_t *sub_e, double *sub_post)
{
    const int N = P->N, M = P->M;
    int iters = 0;
    /* first BP run */
    int ok = bp_run(g, s, lam, o->max_iter, o->variant, o->alpha, 1, e_hat, post, &iters, q, r);
    *it1 = iters; *it2 = 0;
    if (post1) memcpy(post1, post, sizeof(double) * (size_t)N);
    memset(cut, 0, (size_t)N);
    if (ok) return 0;            /* converged: no cut */
    if (!o->dc_enable) return 2;
    /* cut selection */
    oracle_dc_select(P, o, post, shot, cut);
    /* priors of the second run (Sec. III.B): p, or the first-run posterior */
    for (int j = 0; j < N; ++j) {
        if (o->dc_prior == 0) {
            lam2[j] = lam[j];
        } else {
            double ph = 1.0 / (1.0 + exp(post[j]));
            if (ph < 1e-12) ph = 1e-12;
            if (ph > 0.5) ph = 0.5;
            lam2[j] = prior_llr(ph);
        }
    }
    if (o->cut_form == 0) {
        /* second run on the cut graph: DeleteColumns, DeleteEntries, BP, PadWithZeros */
        int nk = 0;
        for (int j = 0; j < N; ++j) keep[j] = cut[j] ? -1 : nk++;
        int ne = 0;
        sub_row_ptr[0] = 0;
        for (int i = 0; i < M; ++i) {
            for (int e = P->h_row_ptr[i]; e < P->h_row_ptr[i + 1]; ++e)
                if (keep[P->h_col[e]] >= 0) sub_col[ne++] = keep[P->h_col[e]];
            sub_row_ptr[i + 1] = ne;
        }
        double *sub_lam = lam2 + N;   /* second half of the scratch */
        for (int j = 0; j < N; ++j) if (keep[j] >= 0) sub_lam[keep[j]] = lam2[j];
        tanner sub;
        tanner_build(&sub, M, nk, sub_row_ptr, sub_col);
        ok = bp_run(&sub, s, sub_lam, o->max_iter, o->variant, o->alpha, 1, sub_e, sub_post, &iters, q, r);
        tanner_free(&sub);
        for (int j = 0; j < N; ++j) {
            e_hat[j] = keep[j] >= 0 ? sub_e[keep[j]] : 0;
            post[j] = keep[j] >= 0 ? sub_post[keep[j]] : INFINITY;
        }
    } else {
        /* Algorithm 2: p_i <- 0 for every cut i, then BP on the full graph */
        for (int j = 0; j < N; ++j) if (cut[j]) lam2[j] = INFINITY;
        ok = bp_run(g, s, lam2, o->max_iter, o->variant, o->alpha, 1, e_hat, post, &iters, q, r);
    }
    *it2 = iters;
    return ok ? 1 : 2;
}

/* Decodes B shots.  syn: B x M bytes (0/1).  Shot b has global index
 * shot_offset + b (it keys the tie-break hash).  Outputs (NULL to skip the
 * optional ones): e_hat B x N bytes, status B bytes, iters1/iters2 B ints,
 * post (final posterior LLR) B x N, post1 (first-run posterior) B x N,
 * cut B x N bytes, obs_pred B x K bytes (e_hat L^T mod 2). */
int oracle_decode_batch(const oracle_problem *P, const oracle_opts *o, int64_t B,
                        const uint8_t *syn, uint64_t shot_offset, uint8_t *e_hat,
                        uint8_t *status, int32_t *iters1, int32_t *iters2, double *post,
                        double *post1, uint8_t *cut, uint8_t *obs_pred, int nthreads)
{
    const int N = P->N, M = P->M, E = P->h_row_ptr[P->M];
    double *lam = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int j = 0; j < N; ++j) lam[j] = prior_llr(P->prior[j]);
    tanner g;
    tanner_build(&g, M, N, P->h_row_ptr, P->h_col);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *q = (double *)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
        double *r = (double *)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
        double *lam2 = (double *)malloc(sizeof(double) * 2 * (size_t)(N > 0 ? N : 1));
        int32_t *keep = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
        int32_t *srp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)M + 1));
        int32_t *scol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
        uint8_t *se = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
        double *sp = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        uint8_t *eh = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
        double *po = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        double *po1 = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        uint8_t *ct = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t b = 0; b < B; ++b) {
            int32_t i1 = 0, i2 = 0;
            int st = decode_shot(P, o, &g, lam, syn + (size_t)b * M, shot_offset + (uint64_t)b,
                                 eh, po, po1, ct, &i1, &i2, q, r, lam2, keep, srp, scol, se, sp);
            if (e_hat) memcpy(e_hat + (size_t)b * N, eh, (size_t)N);
            if (status) status[b] = (uint8_t)st;
            if (iters1) iters1[b] = i1;
            if (iters2) iters2[b] = i2;
            if (post) memcpy(post + (size_t)b * N, po, sizeof(double) * (size_t)N);
            if (post1) memcpy(post1 + (size_t)b * N, po1, sizeof(double) * (size_t)N);
            if (cut) memcpy(cut + (size_t)b * N, ct, (size_t)N);
            if (obs_pred) {
                for (int k = 0; k < P->K; ++k) {
                    int par = 0;
                    for (int a = P->l_row_ptr[k]; a < P->l_row_ptr[k + 1]; ++a) par ^= eh[P->l_col[a]];
                    obs_pred[(size_t)b * P->K + k] = (uint8_t)par;
                }
            }
        }
        free(q); free(r); free(lam2); free(keep); free(srp); free(scol); free(se); free(sp);
        free(eh); free(po); free(po1); free(ct);
    }
    tanner_free(&g);
    free(lam);
    return 0;
}

/* Thread count of the OpenMP loop over shots (n >= 1); timing only. */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
