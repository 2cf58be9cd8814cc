// Internal declarations shared by the host packing code and the CUDA kernels.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace bpdc {

// Check-to-variable magnitudes saturate here; an empty minimum (all other
// neighbours of a check cut) takes this value.
constexpr float kLlrCap = 1e30f;
// Marks an unused check slot (row shorter than the kernel's maximum degree).
constexpr uint16_t kNoEdge = 0xFFFF;
// Limits of the compiled kernel variants.
constexpr int kMaxDRowWeight = 64;

// Message slots per variable pass.  A variant's profile holds 3 bits per pass
// (pass p in bits 3p .. 3p+2, a non-increasing sequence, up to 21 passes):
// pass p gives each of its variables prof_cv slots, so that a graph whose
// variables are sorted by degree into the passes stores no padding for the
// long tail of low-degree columns.  Profile 0: every pass has cv slots.
constexpr int prof_cv(uint64_t prof, int cv, int p) { return prof ? (int)((prof >> (3 * p)) & 0x7u) : cv; }
// Slots of the passes before p (per lane).
constexpr int prof_off(uint64_t prof, int cv, int p)
{
    int s = 0;
    for (int i = 0; i < p; ++i) s += prof_cv(prof, cv, i);
    return s;
}

// Check edges are kept as 16-bit values.  A group whose message slots fit in
// 64 KB of shared memory keeps byte addresses in the block's shared window; a
// larger group (one per block) keeps word indices into its own region and
// scales them when it loads or stores.  slots_per_lane: the variant's slots of
// all passes of one lane.
constexpr bool wide_slots(int G, int slots_per_lane) { return (long)G * slots_per_lane * 4 > 60 * 1024; }
// Check-edge word indices per 16-byte entry of the shared-memory edge table.
constexpr int kTabEdges = 8;

// Device-resident decoding problem, laid out for a group of G threads per
// shot.  Variable j sits at lane j % G, pass j / G; check i at lane i % G,
// pass i / G, except in a shared last check pass (Variant::tail = S lanes per
// check): its c-th check sits on lanes c*S .. c*S+S-1, lane c*S+s holding the
// check's edges s*E .. s*E+E-1 (E = ceil(dc_max / S)) as its entries
// 0 .. E-1 of chk_idx.  Each variable owns `cv` consecutive message slots per pass:
// slot(p, m, u) = (p * cv + m) * G + u holds the message of its m-th edge
// (edges of a variable in ascending check order); unused slots hold 0.
struct DevGraph {
    int32_t M, N, K, Md;
    int32_t MW, NW, KW;          // words per shot of syndrome / correction / logicals
    int32_t G;                   // threads per shot
    int32_t pc, pv;              // check passes, variable passes
    int32_t dc, cv;              // max row weight of H, slots per variable per pass
    int32_t slots;               // pv * cv * G message slots per shot
    int32_t cmw;                 // words of the per-shot variable bit mask (>= NW)
    int32_t region;              // shared-memory words per group
    int32_t max_iter;
    float alpha;
    float tie_rel;
    uint64_t tie_seed;
    int32_t dc_enable, dc_prior;
    int32_t zero_ok;             // every prior < 1/2: zero syndrome decodes to zero at t = 0
    int32_t kernel_id;
    // learned weights of weighted BP (product-sum only), in message-slot order:
    // wts[0][t][slot] scales check -> variable messages, wts[1][t][slot]
    // variable -> check messages of decoding iteration t + 1 (the last set for
    // later iterations); variable -> check messages are clipped to +-w_clip
    const float *wts;            // [2][w_T][slots] or null
    int32_t w_T;
    float w_clip;
    const uint16_t *chk_idx;     // [pc][dc][G] message slot of the check's k-th edge, or kNoEdge
    const uint16_t *chk_word;    // [pc][variant row width][G] the same as word indices of the group's
                                 // region (the +inf word, 2, for none and for padding): read per
                                 // access by the wide kernels
    const uint4 *chk_tab;        // [pc][ceil(row width / 8)][G] the same word indices, 8 per entry
                                 // (edge 8c + e of lane u at pass p in 16-bit half e of entry
                                 // (p, c, u)): copied into shared memory by the wide kernels with an
                                 // edge table
    int32_t tab_off;             // word offset of that shared copy inside the group's region
    const uint8_t *var_deg;      // [pv][G] degree of the variable (0 past N)
    const float *lam;            // [pv][G] prior LLR ln((1-p)/p)
    const int32_t *d_ptr;        // [Md+1] rows of D
    const uint32_t *d_ent;       // [nnz(D)] slot of the variable's first edge | position << 16
    const int32_t *d_col;        // [nnz(D)] column of each D entry (ascending within a row)
    const uint32_t *l_bits;      // [pv*G][KW] columns of L by variable position
    const uint32_t *l_col;       // [N][KW] columns of L by column index (sampler)
    const int32_t *pos_col;      // [pv*G] column of the variable at each position (-1: none)
    const int32_t *h_ptr;        // [M+1] rows of H (sampler)
    const int32_t *h_col;        // [E]
    const uint32_t *thr;         // [N] floor(p * 2^32) (sampler)
    const int32_t *c_ptr;        // [N+1] columns of H: edges of variable j are c_edge[c_ptr[j] .. c_ptr[j+1])
    const int32_t *c_edge;       // [E] edge ids (CSR order of H) by column, ascending check
    const float *lam_col;        // [N] prior LLR by column (weighted BP)
    int32_t *err_flag;           // latched device error code
#ifdef BPDC_CHECKS
    // entries of the tables the checked build compares indices with
    int64_t n_chk_idx, n_chk_word, n_pos, n_d_ent, n_wts;
#endif
};

// One batch of a decode launch (kept in device memory).
struct BatchDesc {
    DevGraph g;
    int64_t B;
    int64_t first;               // prefix of shots of earlier batches in this launch
    const uint32_t *syn;
    uint64_t shot_offset;
    uint32_t *corr;
    uint8_t *status;
    uint32_t *lflips;
    const uint32_t *obs_true;
    uint32_t *iters;
    float *post;
    unsigned long long *counters;
    const uint32_t *cut_in;
};

struct LaunchDesc {
    const BatchDesc *batches;    // device array
    int32_t n_batches;
    int64_t total;               // shots over all batches
    unsigned int *work;          // persistent work counter (nullptr: one group per shot)
};

// A compiled kernel variant and its limits.
struct Variant {
    int id;
    int G;
    int pc_max, dc_max, pv_max, cv_max;
    int cv_min;          // every variable has at least cv_min edges
    bool regular_rows;   // every check has exactly dc_max edges
    int rule;            // check rule: 0 normalized min-sum, 1 product-sum
    int block_threads;
    int min_blocks;      // launch bound: resident blocks per SM the register budget allows
    uint64_t prof;       // slots per variable pass (prof_cv); 0: cv_max in every pass
    bool tab;            // check-edge table in shared memory (wide form only)
    int tail;            // lanes per check of a shared last check pass (0: none; one warp per shot)
};

// Placement of variables on positions and order of the edges inside each
// check (the k of the check update), chosen for conflict-free shared-memory
// access; optimize = false gives the identity placement and CSR order.
struct Layout {
    std::vector<int32_t> pos_of_var;   // [N]
    std::vector<int32_t> var_at_pos;   // [npos], -1 where empty
    std::vector<int32_t> edge_round;   // [nnz(H)] round k of each edge within its check
};
// pass_cv (empty: no limit): slots of each variable pass; a variable of degree
// d then sits in a pass with at least d slots (passes fill in order of
// decreasing degree, so pass_cv must not increase).
void plan_layout(int M, int N, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col, int G,
                 int npos, int dc, bool optimize, const std::vector<int> &pass_cv, Layout &out);

int num_variants();
// Checked builds: the first failed bounds check since the last call (site 0:
// none) and its index, then cleared.  Normal builds return false.
bool check_status(int *site, long long *index);
const Variant &variant(int id);
// Occupancy query and launch of variant `id`.
cudaError_t variant_attributes(int id, int smem_bytes, int *blocks_per_sm, int *regs);
cudaError_t launch_variant(int id, const LaunchDesc &ld, int grid, int smem_bytes, cudaStream_t s);

// Most shots one decode launch takes: the kernel keeps shot indices and work
// tickets in 32 bits (groups of more than 32 threads pass the ticket through a
// 32-bit shared word), and every group draws one ticket past the last shot, so
// every ticket of a launch stays below 2^32 with room for 2^24 groups.
constexpr int64_t kMaxLaunchShots = (int64_t(1) << 32) - (int64_t(1) << 24);

// Largest number of batches one allocation-free launch takes (its scratch is a
// fixed device array).
constexpr int kStaticBatches = 16;
// Launch of variant `id` whose work counter and batch descriptors live in the
// library's fixed device scratch array instead of caller- or library-allocated
// memory.  host_descs: n <= kStaticBatches descriptors in host memory.
cudaError_t launch_variant_static(int id, const BatchDesc *host_descs, int n, int64_t total, int grid,
                                  int smem_bytes, cudaStream_t s);

cudaError_t launch_cut_select(const DevGraph &g, int64_t B, const float *post, uint64_t shot_offset,
                              uint32_t *cut_out, cudaStream_t s);
// Weighted product-sum BP (bpdc_wbp.cu).  Limits: row weight 2..16, column
// weight <= 8; weights W[2][T][E] (E = edges of H in CSR order; W[0] check ->
// variable, W[1] variable -> check).
constexpr int kWbpMaxRow = 16;
constexpr int kWbpMaxCol = 8;
constexpr size_t kMaxWbpSmem = 227 * 1024;
struct WbpArgs {
    int64_t B;
    int E, T, k;                 // edges, iterations, checkpoint interval
    float clip;                  // |q| <= clip
    const uint32_t *syn;         // [B][MW]
    const float *W;              // [2][T][E]
    float *post;                 // [B][T][N] or null
    float *ckpt;                 // [B][ceil(T/k)][E] q of iterations 0, k, 2k, ...
    const float *gpost;          // [B][T][N] adjoint of the posteriors (backward)
    float *part;                 // [B][2][T][E] per-shot gradient partials (backward)
};
size_t wbp_smem_forward(int E, int warps);
size_t wbp_smem_backward(int E, int k, int warps);
cudaError_t launch_wbp_forward(const DevGraph &g, const WbpArgs &a, cudaStream_t s);
cudaError_t launch_wbp_backward(const DevGraph &g, const WbpArgs &a, float *grad_w, cudaStream_t s);

// Shared-memory bandwidth microbenchmark (bpdc_peak.cu): best of three timed
// runs of `reps` iterations on the current device.
cudaError_t measure_smem_peak(int reps, double *bytes_per_s, int *num_sms);
cudaError_t launch_sample(const DevGraph &g, int64_t B, uint64_t seed, uint64_t shot_offset,
                          uint32_t *syn, uint32_t *obs, uint32_t *err, cudaStream_t s);

}  // namespace bpdc
