/*
 * bpdc.h -- C-ABI of the GB300 BP+DC decoder (libbpdc.so).
 *
 * Decodes batches of syndrome shots of one decoding problem (H, L, D, p):
 *   H  (M x N)  matrix whose Tanner graph BP runs on: H_Z under code-capacity
 *               noise, the detector check matrix H_DCM otherwise
 *               (arXiv 2510.08695, Sec. II.C and Sec. IV.A);
 *   L  (K x N)  logical operator matrix O_Z / O, used for the logical flips
 *               e_hat L^T and the failure test (Sec. II.C, Sec. IV.A);
 *   D  (Md x N) degeneracy matrix H_X / H_DDM whose rows degeneracy cutting
 *               acts on (Algorithm 1, Sec. III.A; Sec. IV.B);
 *   p  (N)      prior error probabilities (Eq. 8).
 *
 * The decoder runs flooding BP (Sec. II.C.1) with FP32 messages and the
 * normalized min-sum or the product-sum check rule.  When BP does not reproduce the syndrome within T_iter
 * iterations it cuts, for every row of D, the support variable with the
 * highest posterior LLR (lowest error probability), and runs BP once more on
 * the cut graph with the original priors (Algorithm 1 with the Sec. III.B
 * choice of priors; the cut is applied as in Algorithm 2).
 *
 * Conventions shared by every call:
 *   - Every function returns BPDC_OK (0) or a negative BPDC_ERR_* code and
 *     never aborts the process; bpdc_last_error() gives a message (per
 *     thread).
 *   - Bit vectors are packed little-endian into uint32 words: bit (c % 32) of
 *     word (c / 32) holds entry c.  A shot of a vector of length n takes
 *     ceil(n/32) words; shot b starts at word b * ceil(n/32).
 *   - Device pointers are CUDA device (or managed) addresses on the graph's
 *     device; the caller owns them.  Host pointers are plain host memory.
 *   - Calls taking a stream (cudaStream_t passed as void*, NULL = legacy
 *     default stream) are asynchronous: they only enqueue work.  Argument
 *     errors are reported synchronously; errors raised on the device are
 *     latched in the graph and returned by bpdc_graph_sync_status().
 *   - A graph object may be used from one host thread at a time.  Decode
 *     calls on one graph that run concurrently on different streams are
 *     allowed: each call uses its own slot of the graph's work counters
 *     (at most BPDC_MAX_INFLIGHT calls per graph may be in flight).
 */
#ifndef BPDC_H
#define BPDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BPDC_OK 0
#define BPDC_ERR_INVALID_ARG (-1)   /* a null, out-of-range or inconsistent argument */
#define BPDC_ERR_DIM_MISMATCH (-2)  /* matrix shapes disagree */
#define BPDC_ERR_OOM (-3)           /* device or host allocation failed */
#define BPDC_ERR_CUDA (-4)          /* a CUDA runtime call failed */
#define BPDC_ERR_TIMEOUT (-5)       /* a bounded device-side wait gave up */
#define BPDC_ERR_UNSUPPORTED (-6)   /* valid request the library does not implement */
#define BPDC_ERR_CHECK (-7)         /* checked build: an index left its bounds (access skipped) */

#define BPDC_MAX_INFLIGHT 64

typedef struct bpdc_graph_s *bpdc_graph_t;

/* A 0/1 matrix in CSR form (host memory).  row_ptr has rows+1 entries with
 * row_ptr[0] = 0 and row_ptr[rows] = nnz; col_idx has nnz entries in
 * [0, cols).  Duplicate entries within a row are rejected. */
typedef struct {
    int32_t rows, cols;
    int64_t nnz;
    const int32_t *row_ptr;
    const int32_t *col_idx;
} bpdc_csr;

/* Decoding options, fixed when the graph is created. */
typedef struct {
    int32_t variant;   /* check rule: 0 normalized min-sum, 1 product-sum (Sec. II.C.1
                          cites both; the paper uses product-sum for surface codes) */
    float ms_scale;    /* alpha, the min-sum scale factor, in (0, 1] (unused by product-sum) */
    int32_t max_iter;  /* T_iter, the BP iteration limit of each run, 0..65535 */
    int32_t dc_enable; /* 1: degeneracy cutting on BP failure; 0: plain BP */
    int32_t dc_prior;  /* 0: second BP on the priors p (Sec. III.B, BB codes);
                          1: on the first-run posterior p_hat clamped to
                          [1e-12, 1/2] (Algorithm 1 as printed) */
    float tie_rel;     /* tie window of the cut selection (>= 0): candidates of a
                          row are the variables with
                          L_j >= L_max - tie_rel * max(1, |L_max|) */
    uint64_t tie_seed; /* key of the SplitMix64 tie-break hash: the candidate of
                          rank h(tie_seed, shot * Md + row) mod |candidates|
                          (ascending column order) is cut */
} bpdc_opts;

/* Fills *o with the defaults: min-sum, alpha = 0.625, T_iter = 50, DC on,
 * priors p, tie_rel = 1e-5, tie_seed = 0x2510086950. */
void bpdc_opts_default(bpdc_opts *o);

/* Builds a device-resident decoding problem on CUDA device `device`.
 * H: M x N check matrix (every column must have at least one entry is not
 * required; empty columns are allowed).  L: K x N (K may be 0, rows may be
 * empty).  D: Md x N (Md may be 0; empty rows are skipped by the cut).
 * priors: N host doubles in (0, 1/2].  The library copies everything; the
 * caller may free its arrays on return.  Limits: row weight of D <= 64, and H
 * must fit one compiled kernel variant (bpdc_graph_set_kernel), of which
 * these are the widest:
 *     check rule   M <=   N <=   row weight   column weight
 *     min-sum        96    160   6 exactly    3 exactly     (BB-like, 32 threads)
 *     min-sum       128    256   <= 8         1..4          (32 threads)
 *     min-sum      1536   2560   7 exactly    3..4          (HGP-like)
 *     min-sum      1024   3072   <= 8         2..3          (phenomenological)
 *     min-sum      1024   9216   <= 35        2..6          (circuit-level)
 *     product-sum   128    128   <= 4         1..2          (surface codes)
 *     product-sum    96    160   6 exactly    3 exactly     (BB-like)
 * Larger graphs are UNSUPPORTED.
 * Errors: INVALID_ARG (null pointer, malformed CSR, prior outside (0, 1/2],
 * option out of range), DIM_MISMATCH (column counts differ),
 * UNSUPPORTED (a limit above is exceeded), OOM, CUDA. */
int bpdc_graph_create(const bpdc_csr *H, const bpdc_csr *L, const bpdc_csr *D,
                      const double *priors, const bpdc_opts *opts, int device,
                      bpdc_graph_t *out);

/* Frees the graph and its device memory.  Waits for no stream: the caller
 * must make sure no decode call on the graph is still running.  NULL is a
 * no-op. */
int bpdc_graph_destroy(bpdc_graph_t g);

/* Sizes and the chosen launch plan of a graph. */
typedef struct {
    int32_t M, N, K, Md;
    int64_t E;                  /* nnz(H) = edges of the Tanner graph */
    int32_t syndrome_words;     /* ceil(M/32) */
    int32_t correction_words;   /* ceil(N/32) */
    int32_t logical_words;      /* ceil(K/32) */
    int32_t threads_per_shot;   /* G: threads that decode one shot together */
    int32_t shots_per_block;    /* groups of G threads per CTA */
    int32_t blocks_per_sm;      /* resident CTAs per SM of the persistent form */
    int32_t smem_per_block;     /* dynamic shared memory of one CTA, bytes */
    int32_t kernel_id;          /* index of the compiled kernel variant */
} bpdc_graph_info;

int bpdc_graph_get_info(bpdc_graph_t g, bpdc_graph_info *info);

/* Replaces the launch plan: threads_per_shot G in {4, 8, 16, 32, 64, 128,
 * 256, 512} (0 = automatic).  Used by the autotuner.  UNSUPPORTED if no
 * compiled kernel variant fits the graph with that G. */
int bpdc_graph_set_plan(bpdc_graph_t g, int32_t threads_per_shot);

/* Number of compiled kernel variants (ids 0 .. count-1). */
int bpdc_kernel_count(void);

/* Selects compiled kernel variant `kernel_id` for the graph (the autotuner
 * times every variant that accepts the graph).  INVALID_ARG for an id out of
 * range, UNSUPPORTED if the variant cannot take this graph (group size, row or
 * column weight, regularity or shared-memory limits); the previous plan stays
 * in force on error.  Waits for in-flight decode calls on the graph. */
int bpdc_graph_set_kernel(bpdc_graph_t g, int32_t kernel_id);

/* Message layout of the graph: 1 (the default) places variables and orders
 * the edges of every check so that the check update's shared-memory gathers
 * and scatters avoid bank conflicts; 0 uses the identity placement and the
 * CSR order.  Results are identical; only the speed differs.  Keeps the
 * kernel variant; waits for in-flight decode calls on the graph. */
int bpdc_graph_set_layout(bpdc_graph_t g, int32_t mode);

/* The layout planner alone (host only, no GPU needed): for a check matrix H
 * and a group size G (a multiple of 32) writes the position of every variable
 * (pos_of_var[N], positions in [0, ceil(N/G)*G), bank = pos mod 32) and the
 * round of every edge within its check (edge_round[nnz], in H's CSR order;
 * distinct within a check, below the maximum row weight).  optimize = 0 gives
 * the identity placement and the CSR order. */
int bpdc_layout_plan(const bpdc_csr *H, int32_t G, int32_t optimize, int32_t *pos_of_var, int32_t *edge_round);

/* The same planner under a slot profile (host only; the layouts of the kernel
 * variants whose variable passes have different slot counts):
 * pass_slots[n_pass] (non-increasing, >= 1; n_pass >= ceil(N/G)) gives the
 * message slots of every variable in pass p (positions [p*G, (p+1)*G)); the
 * variables are placed so that each one's column weight is at most its pass's
 * slot count (per bank class, the number of variables of weight >= d stays
 * within the positions of passes with >= d slots; each bank's members fill its
 * positions in order of decreasing weight).  n_pass = 0: no profile (as
 * bpdc_layout_plan).  INVALID_ARG for a malformed profile; UNSUPPORTED when the
 * column weights cannot fit it. */
int bpdc_layout_plan_slots(const bpdc_csr *H, int32_t G, int32_t optimize, int32_t n_pass,
                           const int32_t *pass_slots, int32_t *pos_of_var, int32_t *edge_round);

/* Outputs of a decode call (device pointers; NULL where optional). */
typedef struct {
    uint32_t *corrections;       /* required: [B][ceil(N/32)] e_hat bits (cut variables 0) */
    uint8_t *status;             /* required: [B] 0 BP converged, 1 BP+DC converged, 2 failure */
    uint32_t *logical_flips;     /* optional: [B][ceil(K/32)] bits of e_hat L^T */
    const uint32_t *obs_true;    /* optional input: [B][ceil(K/32)] bits of e L^T of the true
                                    error; with it a shot fails if status == 2 or the
                                    logical flips differ */
    uint32_t *iterations;        /* optional: [B] BP iterations, first run in bits 0-15,
                                    second run in bits 16-31 */
    float *posterior_llr;        /* optional: [B][N] final posterior LLRs (cut variables
                                    +inf); slower path */
    unsigned long long *counters;/* optional: [4] accumulated (atomically added) over the
                                    call: shots, failures (needs obs_true; else status 2),
                                    BP iterations run (both runs), shots that ran DC */
    const uint32_t *cut_in;      /* optional input: [B][ceil(N/32)] a cut set per shot.  With
                                    it the call runs one BP on the cut graph (Algorithm 2
                                    form) and no DC: status 0 converged, 2 not */
} bpdc_outputs;

/* Decodes B >= 0 shots.  syndromes: device [B][ceil(M/32)].  Shot b has the
 * global index shot_offset + b, which keys the tie-break hash, so results do
 * not depend on how shots are split across calls or GPUs.  persistent = 1
 * launches one resident grid that pulls shots from a device work counter;
 * persistent = 0 launches the plain per-batch grid (one group per shot).
 * Both give identical results.  At most 4 278 190 080 (2^32 - 2^24) shots per
 * call (UNSUPPORTED above).  Asynchronous on `stream`. */
int bpdc_decode(bpdc_graph_t g, int64_t B, const uint32_t *syndromes, uint64_t shot_offset,
                const bpdc_outputs *out, int persistent, void *stream);

/* One item of a multi-problem launch. */
typedef struct {
    bpdc_graph_t graph;
    int64_t B;
    const uint32_t *syndromes;
    uint64_t shot_offset;
    bpdc_outputs out;
} bpdc_batch;

/* Decodes several batches, possibly of different graphs, in as few persistent
 * launches as the compiled kernel variants allow (one per variant), with the
 * shots of all batches of a variant behind one device work counter.  All
 * graphs must live on the same device; results equal those of bpdc_decode
 * on each batch.  A launch takes at most 2^32 - 2^24 shots: longer lists are
 * split over several launches, and a single batch above that size is
 * UNSUPPORTED.  Asynchronous on `stream`. */
int bpdc_decode_multi(const bpdc_batch *batches, int32_t n_batches, void *stream);

/* Decoding from host memory (the paper has no counterpart: this is the end-to-
 * end path of a decoder fed by the host).  The same batch list as
 * bpdc_decode_multi, except that syndromes and every output pointer
 * (corrections, status, and if non-NULL logical_flips, obs_true, iterations)
 * are HOST pointers; posterior_llr, counters and cut_in must be NULL
 * (BPDC_ERR_UNSUPPORTED otherwise).  The library cuts every batch into pieces
 * of at most chunk_shots shots (0: 262144) and runs each piece through a
 * three-stage pipeline: copy its syndromes (and obs_true) into one of two
 * device staging sets on a copy stream, decode it with one persistent launch
 * on `stream`, copy its outputs back on a second copy stream, so that the
 * copies of one piece overlap the decoding of its neighbours.  Page-locked
 * host buffers are needed for that overlap (pageable ones give the same
 * results with serialised copies).  The staging memory (two pieces at the
 * widest graph's row widths) is allocated on demand and kept by the first
 * batch's graph until it is destroyed.  Results equal those of
 * bpdc_decode_multi (the tie-break hash keys on the global shot index).
 * Synchronous: returns when every output is in host memory, also after an
 * error; `stream` is left ordered after the last copy. */
int bpdc_decode_host(const bpdc_batch *batches, int32_t n_batches, int64_t chunk_shots, void *stream);

/* Allocation-free variant of bpdc_decode_multi (the paper has no counterpart:
 * this is an integration aid).  Some callers cannot allocate device memory
 * while they decode: a real-time decoding loop that must not stall on the
 * allocator, code embedded in a host framework whose allocator owns all device
 * memory, or a stream that is being captured into a CUDA graph.  This call
 * allocates nothing: the persistent kernel's scratch (its device work counter
 * and the descriptors of up to 16 batches: 256 + 16 x 344 = 5760 bytes) lives in a fixed device
 * array of the library, which every GPU that loads the library holds until the
 * process exits.  The caller still passes every input and output, and the
 * graphs must already exist.
 *   - At most 16 batches per call, all on graphs that use the same kernel
 *     variant (bpdc_graph_info.kernel_id), and at most 2^32 - 2^24 shots in
 *     all; otherwise BPDC_ERR_UNSUPPORTED with a message, and nothing is
 *     launched.
 *   - The first call on a device looks up the array's device address; make
 *     that first call before any stream capture on that device.
 *   - Every call reuses the same array (the work counter is cleared at the
 *     start of each call).  Calls whose launches overlap on the GPU, e.g. on
 *     two streams, race on it: keep such calls ordered on one stream.
 *   - The call issues two kernel launches and nothing else: a setup kernel that
 *     receives the batch descriptors as kernel parameters, writes them into the
 *     array and clears the counter, then the decode kernel.  It can therefore
 *     be captured into a CUDA graph (after a first uncaptured call on the
 *     device); each replay decodes whatever the captured syndrome buffers hold
 *     into the captured output buffers.
 * Results equal those of bpdc_decode_multi on the same batches. */
int bpdc_decode_multi_noalloc(const bpdc_batch *batches, int32_t n_batches, void *stream);

/* Cut selection alone (the selection step of Algorithm 1) from given posterior LLRs:
 * posterior_llr device [B][N] floats, cut_out device [B][ceil(N/32)] bits.
 * Uses the graph's D, tie_rel and tie_seed. */
int bpdc_cut_select(bpdc_graph_t g, int64_t B, const float *posterior_llr, uint64_t shot_offset,
                    uint32_t *cut_out, void *stream);

/* Seeded shot sampler (benchmark inputs): e_ij = [(h(seed, i*N + j) >> 32) <
 * floor(p_j * 2^32)] for global shot i = shot_offset + b, h the SplitMix64
 * output function; writes syndromes e H^T [B][ceil(M/32)] and, if non-NULL,
 * observables e L^T [B][ceil(K/32)] and errors [B][ceil(N/32)]. */
int bpdc_sample(bpdc_graph_t g, int64_t B, uint64_t seed, uint64_t shot_offset,
                uint32_t *syndromes, uint32_t *observables, uint32_t *errors, void *stream);

/* Waits for the graph's device work on `stream` and returns the first device
 * error latched since the last call (BPDC_ERR_TIMEOUT, BPDC_ERR_CUDA), then
 * clears it. */
int bpdc_graph_sync_status(bpdc_graph_t g, void *stream);

/* Failure injection for tests (the paper has none).  After `skip` more
 * allocations, the next `count` device or page-locked allocations that the
 * library makes itself (graph arenas, launch rings and their page-locked
 * descriptor mirrors, host-decode staging) fail as if memory were exhausted,
 * without calling the allocator, so the call making them returns BPDC_ERR_OOM
 * and keeps its graph as it was.  count = 0 turns the injection off.  Process-
 * wide; BPDC_ERR_INVALID_ARG if skip or count is negative. */
int bpdc_debug_fail_allocations(int32_t skip, int32_t count);

/* Bounds checks (a debugging aid; the paper has none).  The library is also
 * built as libbpdc_checked.so with -DBPDC_CHECKS: there the decode kernel
 * compares every shared-memory message access with the block's dynamic shared
 * memory and every read of its per-lane graph tables (check addresses, check
 * words, variable positions, D rows, weights) and every indexed output or
 * cut-mask write with the table's length.  The first violation on a device
 * latches its site (1 shared load, 2 shared store, 3 check-address table,
 * 4 check-word table, 5 position tables, 6 D rows, 7 output / cut-mask index,
 * 8 weights) and index, and the access is skipped; nothing traps.  This call
 * waits for the device, writes the latched site (0: none) and index, clears
 * the latch and returns BPDC_ERR_CHECK if a check failed.  The normal library
 * compiles no checks and returns BPDC_ERR_UNSUPPORTED. */
int bpdc_check_status(int32_t device, int32_t *site, int64_t *index);

/* Shared-memory bandwidth of device `device`, the roof of the decode kernels
 * (their messages stay in shared memory; one 4-byte load and one 4-byte store
 * per message per phase).  Runs a microbenchmark of conflict-free 4-byte
 * loads and stores (8 + 8 per thread and iteration, `reps` iterations,
 * reps >= 8, one wave of as many 1024-thread blocks per SM as fit with 64 KB
 * of shared memory each, about 0.5 us per iteration at 2 GHz) three times
 * after a warm-up run and reports the best rate in bytes per second (CUDA
 * events around the launch; at whatever SM clock the GPU runs then) and the
 * number of SMs.  Synchronous; allocates and frees 4 bytes of device memory.
 * Errors: BPDC_ERR_INVALID_ARG (NULL output, reps < 8), BPDC_ERR_CUDA. */
int bpdc_measure_smem_peak(int32_t device, int32_t reps, double *bytes_per_second, int32_t *num_sms);

/* ---- Weighted BP (differentiable decoding; not part of the paper) ------------
 *
 * Product-sum BP (the check rule Sec. II.C.1 cites) with one weight per edge,
 * iteration and direction, unrolled for exactly T iterations (no early stop,
 * no degeneracy cutting).  Edges e = (i, j) of H are numbered in CSR order
 * (row by row, ascending column).  weights is device float [2][T][E]:
 * W[0][t][e] = wc scales the check-to-variable message, W[1][t][e] = wv the
 * variable-to-check message.  For t = 0..T-1:
 *   q_e(t) = clip(wv[t][e] (lambda_j + sum_{e' in M(j), e' != e} r_e'(t-1)), -clip, clip),  r(-1) = 0
 *   r_e(t) = wc[t][e] (-1)^{s_i} prod_{e' in N(i), e' != e} sgn(q_e'(t))
 *            phi(sum_{e' in N(i), e' != e} phi(max(|q_e'(t)|, 1e-6))),   phi(x) = -log tanh(x/2)
 *   L_j(t) = lambda_j + sum_{e in M(j)} r_e(t)
 * Unit weights and a large clip give the decoder's product-sum BP.  Graphs
 * need row weights 2..16 and column weights <= 8.  The forward keeps the q of
 * iterations 0, k, 2k, ... (k = ckpt_every) in the caller's workspace; the
 * backward recomputes each k-iteration segment from them, so both calls must
 * get the same workspace, weights, syndromes, T, clip and ckpt_every, with the
 * forward first.  Calls are stream-ordered and asynchronous.  Errors:
 * BPDC_ERR_INVALID_ARG (NULL buffers, T outside [1, 1000], ckpt_every
 * outside [1, T], clip outside (0, 30], workspace too small),
 * BPDC_ERR_UNSUPPORTED (row/column weights, or more edges than the adjoint's
 * shared memory holds), BPDC_ERR_CUDA. */

/* Makes bpdc_decode / bpdc_decode_multi run weighted BP with learned weights
 * (host float [2][T][E], the layout above; copied) inside BP+DC: decoding
 * iteration t (t = 1, 2, ...) uses weight set min(t, T) - 1, both BP runs
 * start from set 0, and variable-to-check messages are clipped to +-clip, so
 * that the first T iterations of a run equal bpdc_wbp_forward's.  NULL
 * weights restore plain BP.  The graph must use the product-sum rule
 * (variant 1).  Errors: BPDC_ERR_INVALID_ARG (T outside [1, 1000], clip
 * outside (0, 30], non-finite weight), BPDC_ERR_UNSUPPORTED (min-sum graph),
 * BPDC_ERR_CUDA / BPDC_ERR_OOM (re-upload). */
int bpdc_graph_set_weights(bpdc_graph_t g, const float *weights, int32_t T, float clip);

/* Bytes of workspace the two calls need for B shots. */
int bpdc_wbp_workspace_size(bpdc_graph_t g, int64_t B, int32_t T, int32_t ckpt_every, size_t *bytes);

/* Forward: posterior LLRs of every iteration, device float [B][T][N] (may be
 * NULL when only the checkpoints are wanted).  syndromes: device uint32
 * [B][ceil(M/32)] as for bpdc_decode. */
int bpdc_wbp_forward(bpdc_graph_t g, int64_t B, const uint32_t *syndromes, const float *weights, int32_t T,
                     float clip, int32_t ckpt_every, float *posteriors, void *workspace, size_t workspace_bytes,
                     void *stream);

/* Adjoint: given dLoss/dL_j(t) (device float [B][T][N]), writes
 * dLoss/dW (device float [2][T][E], summed over the B shots in a fixed
 * order, so the result is deterministic). */
int bpdc_decode_backward(bpdc_graph_t g, int64_t B, const uint32_t *syndromes, const float *weights, int32_t T,
                         float clip, int32_t ckpt_every, const float *grad_posteriors, float *grad_weights,
                         void *workspace, size_t workspace_bytes, void *stream);

/* Message of the last error raised on the calling thread ("" if none). */
const char *bpdc_last_error(void);

/* Library version string. */
const char *bpdc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BPDC_H */
