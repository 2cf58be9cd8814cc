// C-ABI of libbpdc.so: argument validation, Tanner-graph packing for the
// group-per-shot kernels, launch planning and asynchronous launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <cmath>
#include <limits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bpdc.h"
#include "bpdc_internal.h"

using namespace bpdc;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(BPDC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Failure injection for tests (bpdc_debug_fail_allocations): after
// g_alloc_skip more allocations, the next g_alloc_fail device or page-locked
// allocations of the library fail as if memory were exhausted.
std::mutex g_alloc_mu;
int g_alloc_skip = 0, g_alloc_fail = 0;

bool injected_alloc_failure()
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_alloc_fail <= 0) return false;
    if (g_alloc_skip > 0) {
        --g_alloc_skip;
        return false;
    }
    --g_alloc_fail;
    return true;
}

cudaError_t lib_malloc(void **p, size_t n)
{
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, n);
}

cudaError_t lib_malloc_host(void **p, size_t n)
{
    if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
    return cudaMallocHost(p, n);
}

// Makes `dev` current for the scope and restores the caller's device.
struct DeviceGuard {
    int old = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&old) != cudaSuccess) old = -1;
        if (old != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (old >= 0) {
            int cur = -1;
            if (cudaGetDevice(&cur) == cudaSuccess && cur != old) cudaSetDevice(old);
        }
    }
};

constexpr int kRing = BPDC_MAX_INFLIGHT;
constexpr int64_t kHostChunk = 262144;   // default shots per piece of bpdc_decode_host
constexpr int kMaxBatches = 32;
constexpr int kMaxSmemPerBlock = 227 * 1024;

struct HostCsr {
    int32_t rows = 0, cols = 0;
    std::vector<int32_t> ptr, col;
};

int copy_csr(const bpdc_csr *m, const char *name, HostCsr &out)
{
    if (!m) return fail(BPDC_ERR_INVALID_ARG, "%s is NULL", name);
    if (m->rows < 0 || m->cols < 0 || m->nnz < 0)
        return fail(BPDC_ERR_INVALID_ARG, "%s has negative dimensions", name);
    if (!m->row_ptr) return fail(BPDC_ERR_INVALID_ARG, "%s.row_ptr is NULL", name);
    if (m->nnz > 0 && !m->col_idx) return fail(BPDC_ERR_INVALID_ARG, "%s.col_idx is NULL", name);
    if (m->row_ptr[0] != 0 || m->row_ptr[m->rows] != m->nnz)
        return fail(BPDC_ERR_INVALID_ARG, "%s.row_ptr must start at 0 and end at nnz", name);
    out.rows = m->rows;
    out.cols = m->cols;
    out.ptr.assign(m->row_ptr, m->row_ptr + m->rows + 1);
    out.col.assign(m->col_idx, m->col_idx + m->nnz);
    for (int32_t r = 0; r < m->rows; ++r) {
        if (out.ptr[r + 1] < out.ptr[r]) return fail(BPDC_ERR_INVALID_ARG, "%s.row_ptr decreases at row %d", name, r);
        std::sort(out.col.begin() + out.ptr[r], out.col.begin() + out.ptr[r + 1]);
        for (int32_t a = out.ptr[r]; a < out.ptr[r + 1]; ++a) {
            if (out.col[a] < 0 || out.col[a] >= m->cols)
                return fail(BPDC_ERR_INVALID_ARG, "%s: column %d out of range in row %d", name, out.col[a], r);
            if (a > out.ptr[r] && out.col[a] == out.col[a - 1])
                return fail(BPDC_ERR_INVALID_ARG, "%s: duplicate column %d in row %d", name, out.col[a], r);
        }
    }
    return BPDC_OK;
}

struct RingSlot {
    BatchDesc *dev_desc = nullptr;       // kMaxBatches descriptors
    BatchDesc *host_desc = nullptr;      // pinned mirror
    unsigned long long *work = nullptr;  // persistent work counter
    cudaEvent_t done = nullptr;
    bool used = false;
};

}  // namespace

struct bpdc_graph_s {
    int device = 0;
    int sm_count = 0;
    bpdc_opts opts{};
    HostCsr H, L, D;
    std::vector<double> priors;
    DevGraph dg{};
    void *arena = nullptr;
    int variant = -1;
    int groups_per_block = 0;
    int blocks_per_sm = 0;
    int smem_bytes = 0;
    int regs = 0;
    void *ring_mem = nullptr;
    void *ring_host = nullptr;
    RingSlot ring[kRing];
    int ring_next = 0;
    int layout = 1;   // 1: bank-conflict-aware placement, 0: identity
    std::vector<float> w_host;   // learned weights [2][w_T][E] (CSR edge order), empty if none
    int w_T = 0;
    float w_clip = 0.0f;
    // decoding from host buffers (bpdc_decode_host): two device staging sets,
    // the copy streams, and the events that order copies against decodes
    void *stage = nullptr;
    size_t stage_set_bytes = 0;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_dec[2] = {}, ev_out[2] = {};
    cudaEvent_t ev_entry = nullptr, ev_exit = nullptr;
    std::mutex mu;
};

namespace {

// Message-slot layout of the packing: variable j at lane j % G, pass j / G,
// its m-th edge (ascending check index) in slot ((j/G)*cv + m)*G + j%G.
struct Packed {
    int G, pc, pv, dc, cv, slots, cmw, region, KW, NW, MW, tab_off;
    std::vector<int> pass_off;   // [pv + 1] slots (per lane) before each pass
    std::vector<uint16_t> chk_idx;
    std::vector<uint16_t> chk_word;
    std::vector<uint16_t> chk_tab;   // [ceil(row width / 8)][G][8] (wide variants with a table)
    std::vector<uint8_t> var_deg;
    std::vector<float> lam;
    std::vector<int32_t> d_ptr;
    std::vector<uint32_t> d_ent;
    std::vector<int32_t> d_col;
    std::vector<uint32_t> l_pos;
    std::vector<uint32_t> l_cols;
    std::vector<uint32_t> thr;
    std::vector<int32_t> pos_col;
    std::vector<float> wts;      // [2][w_T][slots] (empty without weights)
};

// Packs the graph for kernel variant v; returns false if v cannot take it.
bool pack(const bpdc_graph_s &g, const Variant &v, Packed &P)
{
    const int G = v.G;
    const int M = g.H.rows, N = g.H.cols, K = g.L.rows, Md = g.D.rows;
    P.G = G;
    P.pc = std::max(1, (M + G - 1) / G);
    P.pv = std::max(1, (N + G - 1) / G);
    std::vector<int> deg(N, 0);
    int dmax = 0, dmin = M > 0 ? 1 << 30 : 0;
    for (int i = 0; i < M; ++i) {
        const int d = g.H.ptr[i + 1] - g.H.ptr[i];
        dmax = std::max(dmax, d);
        dmin = std::min(dmin, d);
    }
    for (int32_t c : g.H.col) deg[c]++;
    int cmax = 0, cmin = N > 0 ? 1 << 30 : 0;
    for (int j = 0; j < N; ++j) {
        cmax = std::max(cmax, deg[j]);
        cmin = std::min(cmin, deg[j]);
    }
    if (v.rule != g.opts.variant) return false;
    if (P.pc > v.pc_max || P.pv > v.pv_max || dmax > v.dc_max || cmax > v.cv_max) return false;
    if (v.regular_rows && (dmin != v.dc_max || dmax != v.dc_max)) return false;
    if (cmin < v.cv_min) return false;
    // a shared last check pass (regular rows only) holds G / tail checks
    const bool tail = v.tail > 0 && P.pc == v.pc_max;
    if (v.tail > 0 && (!v.regular_rows || (tail && M - (P.pc - 1) * G > G / v.tail))) return false;
    P.dc = std::max(dmax, 1);
    P.cv = v.cv_max;
    // slots per pass (the variant's profile), and the degrees it can hold
    std::vector<int> pass_cv(P.pv);
    P.pass_off.assign(P.pv + 1, 0);
    for (int p = 0; p < P.pv; ++p) {
        pass_cv[p] = prof_cv(v.prof, v.cv_max, p);
        P.pass_off[p + 1] = P.pass_off[p] + pass_cv[p];
    }
    if (v.prof) {
        // with degrees sorted into the passes, the i-th largest degree must fit
        // the pass of position i
        std::vector<int> ds(deg);
        std::sort(ds.begin(), ds.end(), std::greater<int>());
        for (int j = 0; j < N; ++j)
            if (ds[j] > pass_cv[j / G]) return false;
    }
    const long slots = (long)P.pass_off[P.pv] * G;
    if (slots > 65535) return false;
    P.slots = (int)slots;
    P.cmw = (P.pv * G + 31) / 32;
    P.NW = (N + 31) / 32;
    P.MW = (M + 31) / 32;
    P.KW = (K + 31) / 32;
    int region = 12 + P.slots + P.cmw + std::max(P.KW, 1);   // 12 misc words (see the kernels)
    region = (region + 3) & ~3;
    // the wide form with an edge table keeps each lane's check-edge word
    // indices in shared memory after the group's other words (16-byte entries)
    const int tab_chunks = (std::max(v.dc_max, P.dc) + kTabEdges - 1) / kTabEdges;
    P.tab_off = 0;
    if (v.tab) {   // one 16-byte entry per 8 edges of every check pass of a lane
        P.tab_off = region;
        region += P.pc * tab_chunks * G * 4;
    }
    P.region = region;
    // check edges are kept as 16-bit values in the kernels: byte addresses
    // below 64 KB (the block's dynamic shared memory plus the reserved 1 KB),
    // or, in the wide form, word indices of the group's region
    if (wide_slots(G, prof_off(v.prof, v.cv_max, v.pv_max))) {
        if (12 + P.slots + P.cmw > 65535 || (long)(v.block_threads / G) * region * 4 > kMaxSmemPerBlock) return false;
    } else if (v.tab || (long)(v.block_threads / G) * region * 4 + 1024 > 65535) {
        return false;
    }
    // variable placement and edge order (bpdc_layout.cu)
    const int npos = P.pv * G;
    Layout lay;
    plan_layout(M, N, g.H.ptr, g.H.col, G, npos, P.dc, g.layout != 0, pass_cv, lay);
    for (int j = 0; j < N; ++j)
        if (deg[j] > pass_cv[lay.pos_of_var[j] / G]) return false;
    // edge -> slot of its variable
    std::vector<int> fill(N, 0);
    std::vector<int> edge_slot(g.H.col.size());
    for (int i = 0; i < M; ++i)
        for (int a = g.H.ptr[i]; a < g.H.ptr[i + 1]; ++a) {
            const int j = g.H.col[a];
            const int pos = lay.pos_of_var[j];
            const int m = fill[j]++;
            edge_slot[a] = (P.pass_off[pos / G] + m) * G + (pos % G);
        }
    if (!g.w_host.empty()) {   // learned weights into message-slot order
        const size_t E = g.H.col.size();
        P.wts.assign((size_t)2 * g.w_T * P.slots, 1.0f);
        for (int h = 0; h < 2 * g.w_T; ++h)
            for (size_t a = 0; a < E; ++a) P.wts[(size_t)h * P.slots + edge_slot[a]] = g.w_host[h * E + a];
    }
    P.chk_idx.assign((size_t)P.pc * P.dc * G, kNoEdge);
    const int tail_e = v.tail > 0 ? (v.dc_max + v.tail - 1) / v.tail : 0;   // edges per lane in it
    for (int i = 0; i < M; ++i) {
        const int p = i / G, u = i % G;
        for (int a = g.H.ptr[i]; a < g.H.ptr[i + 1]; ++a) {
            const int r = lay.edge_round[a];
            if (tail && p == P.pc - 1)   // edge r of the pass's u-th check: lane u*tail + r/E, entry r%E
                P.chk_idx[((size_t)p * P.dc + r % tail_e) * G + u * v.tail + r / tail_e] = (uint16_t)edge_slot[a];
            else
                P.chk_idx[((size_t)p * P.dc + r) * G + u] = (uint16_t)edge_slot[a];
        }
    }
    // the same edges as word indices of the group's region (12 misc words
    // first; 2 = the +inf word), with the variant's full row width per pass
    // so that a kernel reads every entry of its compile-time width in bounds
    {
        const int dcw = std::max(v.dc_max, P.dc);
        P.chk_word.assign((size_t)P.pc * dcw * G, (uint16_t)2);
        for (int p = 0; p < P.pc; ++p)
            for (int k = 0; k < P.dc; ++k)
                for (int u = 0; u < G; ++u) {
                    const uint16_t e = P.chk_idx[((size_t)p * P.dc + k) * G + u];
                    if (e != kNoEdge) P.chk_word[((size_t)p * dcw + k) * G + u] = (uint16_t)(12 + e);
                }
        if (v.tab) {
            // 8 edges of one lane per 16-byte entry: entry (p, c, u) holds edges
            // 8c .. 8c+7 of lane u at check pass p, padded with the +inf word
            P.chk_tab.assign((size_t)P.pc * tab_chunks * G * kTabEdges, (uint16_t)2);
            for (int p = 0; p < P.pc; ++p)
                for (int k = 0; k < std::min(dcw, tab_chunks * kTabEdges); ++k)
                    for (int u = 0; u < G; ++u)
                        P.chk_tab[(((size_t)p * tab_chunks + k / kTabEdges) * G + u) * kTabEdges + k % kTabEdges] =
                            P.chk_word[((size_t)p * dcw + k) * G + u];
        }
    }
    P.var_deg.assign((size_t)npos, 0xFF);   // 0xFF: no variable at this position
    P.lam.assign((size_t)npos, std::numeric_limits<float>::infinity());
    P.pos_col.assign((size_t)npos, -1);
    for (int j = 0; j < N; ++j) {
        const int pos = lay.pos_of_var[j];
        P.var_deg[pos] = (uint8_t)deg[j];
        // The decoder keeps each variable's hard decision in the mantissa LSB
        // of the messages it sends.  Priors are stored with that bit clear,
        // so the first messages carry lambda unchanged and exact identities
        // of the rule (lambda - lambda = 0 through a two-input check) are
        // not moved off zero by the tag; the change is at most one ulp.
        float lam = (float)std::log((1.0 - g.priors[j]) / g.priors[j]);
        uint32_t lb;
        std::memcpy(&lb, &lam, 4);
        lb &= ~1u;
        std::memcpy(&lam, &lb, 4);
        P.lam[pos] = lam;
        P.pos_col[pos] = j;
    }
    P.d_ptr.assign(Md + 1, 0);
    P.d_ent.clear();
    P.d_col.clear();
    for (int r = 0; r < Md; ++r) {
        for (int a = g.D.ptr[r]; a < g.D.ptr[r + 1]; ++a) {
            const int j = g.D.col[a];
            const int pos = lay.pos_of_var[j];
            // slot of the variable's first edge (it holds L after the last
            // iteration); kNoEdge for a variable without edges (L = lambda)
            const uint32_t s0 = deg[j] > 0 ? (uint32_t)(P.pass_off[pos / G] * G + (pos % G)) : kNoEdge;
            P.d_ent.push_back(s0 | ((uint32_t)pos << 16));
            P.d_col.push_back(j);
        }
        P.d_ptr[r + 1] = (int32_t)P.d_ent.size();
    }
    const int kw = std::max(P.KW, 1);
    P.l_cols.assign((size_t)N * kw, 0);
    P.l_pos.assign((size_t)npos * kw, 0);
    for (int k = 0; k < K; ++k)
        for (int a = g.L.ptr[k]; a < g.L.ptr[k + 1]; ++a) {
            const int j = g.L.col[a];
            P.l_cols[(size_t)j * kw + (k >> 5)] |= 1u << (k & 31);
            P.l_pos[(size_t)lay.pos_of_var[j] * kw + (k >> 5)] |= 1u << (k & 31);
        }
    P.thr.resize(N);
    for (int j = 0; j < N; ++j) P.thr[j] = (uint32_t)std::floor(g.priors[j] * 4294967296.0);
    return true;
}

template <typename T>
size_t put(std::vector<char> &blob, const std::vector<T> &v)
{
    size_t off = (blob.size() + 255) & ~(size_t)255;
    blob.resize(off + std::max<size_t>(v.size() * sizeof(T), 4), 0);
    if (!v.empty()) memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

// Packs the graph for threads_per_shot G (0 = automatic) and uploads it.
int plan_and_upload(bpdc_graph_s *g, int want_G, int want_id = -1)
{
    // automatic preference: one warp per shot for small graphs (3 blocks per
    // SM before 4: the same speed with fewer spills; a shared last check pass
    // before the plain form of the same shape), then the 256- and 512-thread
    // groups (a slot-profile variant before the uniform one of the same shape:
    // it is faster wherever its profile fits the graph)
    static const int kOrder[] = {19, 17, 20, 7, 0, 12, 5, 11, 15, 1, 3, 2, 4, 6, 16, 14, 13, 18};
    Packed P{};
    int vid = -1;
    for (int id : kOrder) {
        if (id >= num_variants()) continue;
        const Variant &v = variant(id);
        if (want_G && v.G != want_G) continue;
        Packed Q{};
        if (pack(*g, v, Q)) { P = std::move(Q); vid = id; break; }
    }
    if (want_id >= 0) {
        vid = -1;
        Packed Q{};
        if (want_id < num_variants() && pack(*g, variant(want_id), Q)) { P = std::move(Q); vid = want_id; }
    }
    if (vid < 0)
        return fail(BPDC_ERR_UNSUPPORTED, "no compiled kernel variant fits this graph%s",
                    want_G ? " with the requested threads per shot" : "");
    const Variant &v = variant(vid);
    const int gpb = v.block_threads / v.G;
    const int smem = gpb * P.region * 4;
    int bps = 0, regs = 0;
    cudaError_t e = variant_attributes(vid, smem, &bps, &regs);
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    if (bps < 1) return fail(BPDC_ERR_UNSUPPORTED, "kernel variant %d cannot be resident with %d bytes of shared memory", vid, smem);

    // device arena
    std::vector<char> blob;
    const size_t o_chk = put(blob, P.chk_idx), o_deg = put(blob, P.var_deg), o_lam = put(blob, P.lam);
    const size_t o_chkw = put(blob, P.chk_word), o_tab = put(blob, P.chk_tab);
    const size_t o_dptr = put(blob, P.d_ptr), o_dent = put(blob, P.d_ent), o_l = put(blob, P.l_pos);
    const size_t o_dcol = put(blob, P.d_col), o_lcol = put(blob, P.l_cols), o_pcol = put(blob, P.pos_col);
    const size_t o_hptr = put(blob, g->H.ptr), o_hcol = put(blob, g->H.col), o_thr = put(blob, P.thr);
    // column view of H and priors by column (weighted BP)
    std::vector<int32_t> cptr(g->H.cols + 1, 0), cedge(g->H.col.size());
    std::vector<float> lamc(g->H.cols);
    for (int32_t c : g->H.col) cptr[c + 1]++;
    for (int j = 0; j < g->H.cols; ++j) cptr[j + 1] += cptr[j];
    {
        std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
        for (int i = 0; i < g->H.rows; ++i)
            for (int a = g->H.ptr[i]; a < g->H.ptr[i + 1]; ++a) cedge[fill[g->H.col[a]]++] = a;
        for (int j = 0; j < g->H.cols; ++j)
            lamc[j] = (float)std::log((1.0 - g->priors[j]) / g->priors[j]);
    }
    const size_t o_cptr = put(blob, cptr), o_cedge = put(blob, cedge), o_lamc = put(blob, lamc);
    const size_t o_wts = put(blob, P.wts);
    const size_t o_err = put(blob, std::vector<int32_t>(4, 0));
    void *arena = nullptr;
    e = lib_malloc(&arena, blob.size());
    if (e != cudaSuccess) return fail(BPDC_ERR_OOM, "cudaMalloc of %zu bytes: %s", blob.size(), cudaGetErrorString(e));
    e = cudaMemcpy(arena, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(arena); return cuda_fail(e, "upload of the graph"); }
    if (g->arena) cudaFree(g->arena);
    g->arena = arena;
    char *base = (char *)arena;
    DevGraph &d = g->dg;
    d.M = g->H.rows; d.N = g->H.cols; d.K = g->L.rows; d.Md = g->D.rows;
    d.MW = P.MW; d.NW = P.NW; d.KW = P.KW;
    d.G = P.G; d.pc = P.pc; d.pv = P.pv; d.dc = P.dc; d.cv = P.cv;
    d.slots = P.slots; d.cmw = P.cmw; d.region = P.region;
    d.max_iter = g->opts.max_iter;
    d.alpha = g->opts.ms_scale;
    d.tie_rel = g->opts.tie_rel;
    d.tie_seed = g->opts.tie_seed;
    d.dc_enable = g->opts.dc_enable;
    d.dc_prior = g->opts.dc_prior;
    d.zero_ok = 1;
    for (double p : g->priors) if (!(p < 0.5)) d.zero_ok = 0;
    d.kernel_id = vid;
    d.chk_idx = (const uint16_t *)(base + o_chk);
    d.chk_word = (const uint16_t *)(base + o_chkw);
    d.chk_tab = (const uint4 *)(base + o_tab);
    d.tab_off = P.tab_off;
    d.var_deg = (const uint8_t *)(base + o_deg);
    d.lam = (const float *)(base + o_lam);
    d.d_ptr = (const int32_t *)(base + o_dptr);
    d.d_ent = (const uint32_t *)(base + o_dent);
    d.l_bits = (const uint32_t *)(base + o_l);
    d.d_col = (const int32_t *)(base + o_dcol);
    d.l_col = (const uint32_t *)(base + o_lcol);
    d.pos_col = (const int32_t *)(base + o_pcol);
    d.h_ptr = (const int32_t *)(base + o_hptr);
    d.h_col = (const int32_t *)(base + o_hcol);
    d.thr = (const uint32_t *)(base + o_thr);
    d.c_ptr = (const int32_t *)(base + o_cptr);
    d.c_edge = (const int32_t *)(base + o_cedge);
    d.lam_col = (const float *)(base + o_lamc);
    d.wts = P.wts.empty() ? nullptr : (const float *)(base + o_wts);
    d.w_T = P.wts.empty() ? 0 : g->w_T;
    d.w_clip = g->w_clip;
    d.err_flag = (int32_t *)(base + o_err);
#ifdef BPDC_CHECKS
    d.n_chk_idx = (int64_t)P.chk_idx.size();
    d.n_chk_word = (int64_t)P.chk_word.size();
    d.n_pos = (int64_t)P.pos_col.size();
    d.n_d_ent = (int64_t)P.d_ent.size();
    d.n_wts = (int64_t)P.wts.size();
#endif
    g->variant = vid;
    g->groups_per_block = gpb;
    g->blocks_per_sm = bps;
    g->smem_bytes = smem;
    g->regs = regs;
    return BPDC_OK;
}

int ring_init(bpdc_graph_s *g)
{
    const size_t per = sizeof(BatchDesc) * kMaxBatches + 256;
    cudaError_t e = lib_malloc(&g->ring_mem, per * kRing);
    if (e != cudaSuccess) return fail(BPDC_ERR_OOM, "ring allocation: %s", cudaGetErrorString(e));
    e = lib_malloc_host(&g->ring_host, sizeof(BatchDesc) * kMaxBatches * kRing);
    if (e != cudaSuccess) return fail(BPDC_ERR_OOM, "pinned ring allocation: %s", cudaGetErrorString(e));
    for (int s = 0; s < kRing; ++s) {
        char *b = (char *)g->ring_mem + per * s;
        g->ring[s].work = (unsigned long long *)b;
        g->ring[s].dev_desc = (BatchDesc *)(b + 256);
        g->ring[s].host_desc = (BatchDesc *)g->ring_host + (size_t)kMaxBatches * s;
        e = cudaEventCreateWithFlags(&g->ring[s].done, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "event creation");
    }
    return BPDC_OK;
}

void graph_free(bpdc_graph_s *g)
{
    for (int s = 0; s < kRing; ++s)
        if (g->ring[s].done) cudaEventDestroy(g->ring[s].done);
    for (int k = 0; k < 2; ++k) {
        if (g->ev_in[k]) cudaEventDestroy(g->ev_in[k]);
        if (g->ev_dec[k]) cudaEventDestroy(g->ev_dec[k]);
        if (g->ev_out[k]) cudaEventDestroy(g->ev_out[k]);
    }
    if (g->ev_entry) cudaEventDestroy(g->ev_entry);
    if (g->ev_exit) cudaEventDestroy(g->ev_exit);
    if (g->copy_in) cudaStreamDestroy(g->copy_in);
    if (g->copy_out) cudaStreamDestroy(g->copy_out);
    if (g->stage) cudaFree(g->stage);
    if (g->ring_mem) cudaFree(g->ring_mem);
    if (g->ring_host) cudaFreeHost(g->ring_host);
    if (g->arena) cudaFree(g->arena);
    delete g;
}

int check_outputs(const bpdc_outputs *o)
{
    if (!o) return fail(BPDC_ERR_INVALID_ARG, "outputs is NULL");
    if (!o->corrections) return fail(BPDC_ERR_INVALID_ARG, "outputs.corrections is NULL");
    if (!o->status) return fail(BPDC_ERR_INVALID_ARG, "outputs.status is NULL");
    return BPDC_OK;
}

void fill_desc(BatchDesc &d, const bpdc_graph_s *g, int64_t B, const uint32_t *syn, uint64_t off,
               const bpdc_outputs *o, int64_t first)
{
    d.g = g->dg;
    d.B = B;
    d.first = first;
    d.syn = syn;
    d.shot_offset = off;
    d.corr = o->corrections;
    d.status = o->status;
    d.lflips = o->logical_flips;
    d.obs_true = o->obs_true;
    d.iters = o->iterations;
    d.post = o->posterior_llr;
    d.counters = o->counters;
    d.cut_in = o->cut_in;
}

// Enqueues one launch of variant `vid` over n descriptors (already filled in
// the host mirror of ring slot s).
int enqueue(bpdc_graph_s *g, int s, int n, int64_t total, int vid, int smem, bool persistent,
            cudaStream_t stream)
{
    if (total > kMaxLaunchShots)
        return fail(BPDC_ERR_UNSUPPORTED, "at most %lld shots per launch (got %lld)", (long long)kMaxLaunchShots,
                    (long long)total);
    RingSlot &rs = g->ring[s];
    cudaError_t e = cudaMemcpyAsync(rs.dev_desc, rs.host_desc, sizeof(BatchDesc) * n,
                                    cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "descriptor upload");
    LaunchDesc ld{};
    ld.batches = rs.dev_desc;
    ld.n_batches = n;
    ld.total = total;
    ld.work = nullptr;
    const Variant &v = variant(vid);
    const int gpb = v.block_threads / v.G;
    int bps = 0, regs = 0;
    e = variant_attributes(vid, smem, &bps, &regs);
    if (e != cudaSuccess) return cuda_fail(e, "kernel attributes");
    if (bps < 1) return fail(BPDC_ERR_UNSUPPORTED, "kernel variant %d not resident with %d bytes", vid, smem);
    int64_t grid;
    const int64_t need = (total + gpb - 1) / gpb;
    if (persistent) {
        e = cudaMemsetAsync(rs.work, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return cuda_fail(e, "work counter reset");
        ld.work = (unsigned int *)rs.work;
        grid = std::min<int64_t>((int64_t)g->sm_count * bps, need);
    } else {
        grid = need;
    }
    if (grid > 0x7FFFFFFF) return fail(BPDC_ERR_UNSUPPORTED, "batch too large for one launch");
    e = launch_variant(vid, ld, (int)grid, smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    e = cudaEventRecord(rs.done, stream);
    if (e != cudaSuccess) return cuda_fail(e, "event record");
    rs.used = true;
    return BPDC_OK;
}

int acquire_slot(bpdc_graph_s *g)
{
    const int s = g->ring_next;
    g->ring_next = (g->ring_next + 1) % kRing;
    if (g->ring[s].used) cudaEventSynchronize(g->ring[s].done);
    return s;
}

}  // namespace

extern "C" {

void bpdc_opts_default(bpdc_opts *o)
{
    if (!o) return;
    o->variant = 0;
    o->ms_scale = 0.625f;
    o->max_iter = 50;
    o->dc_enable = 1;
    o->dc_prior = 0;
    o->tie_rel = 1e-5f;
    o->tie_seed = 0x2510086950ull;
}

const char *bpdc_last_error(void) { return g_last_error.c_str(); }

const char *bpdc_version(void) { return "bpdc 0.1 (sm_103a)"; }

int bpdc_graph_create(const bpdc_csr *H, const bpdc_csr *L, const bpdc_csr *D, const double *priors,
                      const bpdc_opts *opts, int device, bpdc_graph_t *out)
{
    g_last_error.clear();
    if (!out) return fail(BPDC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!priors) return fail(BPDC_ERR_INVALID_ARG, "priors is NULL");
    bpdc_opts o;
    if (opts) o = *opts; else bpdc_opts_default(&o);
    if (o.variant != 0 && o.variant != 1)
        return fail(BPDC_ERR_INVALID_ARG, "variant must be 0 (min-sum) or 1 (product-sum)");
    if (!(o.ms_scale > 0.0f && o.ms_scale <= 1.0f)) return fail(BPDC_ERR_INVALID_ARG, "ms_scale must be in (0, 1]");
    if (o.max_iter < 0 || o.max_iter > 65535) return fail(BPDC_ERR_INVALID_ARG, "max_iter must be in [0, 65535]");
    if ((o.dc_enable != 0 && o.dc_enable != 1) || (o.dc_prior != 0 && o.dc_prior != 1))
        return fail(BPDC_ERR_INVALID_ARG, "dc_enable and dc_prior must be 0 or 1");
    if (!(o.tie_rel >= 0.0f) || !std::isfinite(o.tie_rel)) return fail(BPDC_ERR_INVALID_ARG, "tie_rel must be finite and >= 0");
    auto *g = new (std::nothrow) bpdc_graph_s();
    if (!g) return fail(BPDC_ERR_OOM, "host allocation");
    g->opts = o;
    g->device = device;
    int rc;
    if ((rc = copy_csr(H, "H", g->H)) != BPDC_OK || (rc = copy_csr(L, "L", g->L)) != BPDC_OK ||
        (rc = copy_csr(D, "D", g->D)) != BPDC_OK) {
        delete g;
        return rc;
    }
    const int N = g->H.cols;
    if (g->L.cols != N || g->D.cols != N) {
        delete g;
        return fail(BPDC_ERR_DIM_MISMATCH, "H, L and D must have the same number of columns (%d, %d, %d)", N,
                    g->L.cols, g->D.cols);
    }
    if (N > 65535 || g->H.rows > 65535) {
        delete g;
        return fail(BPDC_ERR_UNSUPPORTED, "at most 65535 variables and checks");
    }
    for (int r = 0; r < g->D.rows; ++r)
        if (g->D.ptr[r + 1] - g->D.ptr[r] > kMaxDRowWeight) {
            delete g;
            return fail(BPDC_ERR_UNSUPPORTED, "row %d of D has weight above %d", r, kMaxDRowWeight);
        }
    g->priors.assign(priors, priors + N);
    for (int j = 0; j < N; ++j)
        if (!(g->priors[j] > 0.0 && g->priors[j] <= 0.5)) {
            delete g;
            return fail(BPDC_ERR_INVALID_ARG, "prior %d = %g outside (0, 1/2]", j, g->priors[j]);
        }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "cudaGetDeviceCount"); }
    if (device < 0 || device >= ndev) { delete g; return fail(BPDC_ERR_INVALID_ARG, "device %d does not exist", device); }
    DeviceGuard dgd(device);
    if (!dgd.ok) { delete g; return fail(BPDC_ERR_CUDA, "cannot select device %d", device); }
    e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) { delete g; return cuda_fail(e, "SM count"); }
    if ((rc = plan_and_upload(g, 0)) != BPDC_OK || (rc = ring_init(g)) != BPDC_OK) {
        graph_free(g);
        return rc;
    }
    *out = g;
    return BPDC_OK;
}

int bpdc_graph_destroy(bpdc_graph_t g)
{
    if (!g) return BPDC_OK;
    DeviceGuard dgd(g->device);
    graph_free(g);
    return BPDC_OK;
}

int bpdc_graph_get_info(bpdc_graph_t g, bpdc_graph_info *info)
{
    if (!g || !info) return fail(BPDC_ERR_INVALID_ARG, "NULL argument");
    info->M = g->dg.M; info->N = g->dg.N; info->K = g->dg.K; info->Md = g->dg.Md;
    info->E = (int64_t)g->H.col.size();
    info->syndrome_words = g->dg.MW;
    info->correction_words = g->dg.NW;
    info->logical_words = g->dg.KW;
    info->threads_per_shot = g->dg.G;
    info->shots_per_block = g->groups_per_block;
    info->blocks_per_sm = g->blocks_per_sm;
    info->smem_per_block = g->smem_bytes;
    info->kernel_id = g->variant;
    return BPDC_OK;
}

static int replan(bpdc_graph_t g, int want_G, int want_id)
{
    std::lock_guard<std::mutex> lk(g->mu);
    DeviceGuard dgd(g->device);
    // wait for launches that still read the old arena
    for (int s = 0; s < kRing; ++s)
        if (g->ring[s].used) cudaEventSynchronize(g->ring[s].done);
    const DevGraph keep = g->dg;
    void *keep_arena = g->arena;
    const int kv = g->variant, kg = g->groups_per_block, kb = g->blocks_per_sm, ks = g->smem_bytes;
    g->arena = nullptr;
    int rc = plan_and_upload(g, want_G, want_id);
    if (rc != BPDC_OK) {
        g->dg = keep; g->arena = keep_arena; g->variant = kv;
        g->groups_per_block = kg; g->blocks_per_sm = kb; g->smem_bytes = ks;
        return rc;
    }
    cudaFree(keep_arena);
    return BPDC_OK;
}

int bpdc_graph_set_plan(bpdc_graph_t g, int32_t threads_per_shot)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    static const int ok[] = {0, 4, 8, 16, 32, 64, 128, 256, 512};
    if (std::find(std::begin(ok), std::end(ok), threads_per_shot) == std::end(ok))
        return fail(BPDC_ERR_INVALID_ARG, "threads_per_shot %d not in {0,4,...,512}", threads_per_shot);
    return replan(g, threads_per_shot, -1);
}

int bpdc_kernel_count(void) { return num_variants(); }

int bpdc_layout_plan_slots(const bpdc_csr *H, int32_t G, int32_t optimize, int32_t n_pass, const int32_t *pass_slots,
                           int32_t *pos_of_var, int32_t *edge_round)
{
    HostCsr h;
    int rc = copy_csr(H, "H", h);
    if (rc != BPDC_OK) return rc;
    if (G < 32 || G % 32 != 0 || G > 1024) return fail(BPDC_ERR_INVALID_ARG, "G must be a multiple of 32 in [32, 1024]");
    if (!pos_of_var || !edge_round) return fail(BPDC_ERR_INVALID_ARG, "NULL output");
    const int pv = std::max(1, (h.cols + G - 1) / G);
    std::vector<int> pass_cv;
    std::vector<int> deg(h.cols, 0);
    for (int32_t c : h.col) deg[c]++;
    if (n_pass > 0) {
        if (!pass_slots) return fail(BPDC_ERR_INVALID_ARG, "pass_slots is NULL");
        if (n_pass < pv) return fail(BPDC_ERR_INVALID_ARG, "%d passes cannot hold %d variables at G = %d", n_pass, h.cols, G);
        for (int p = 0; p < pv; ++p) {
            if (pass_slots[p] < 1 || (p > 0 && pass_slots[p] > pass_slots[p - 1]))
                return fail(BPDC_ERR_INVALID_ARG, "pass_slots must be positive and non-increasing");
            pass_cv.push_back(pass_slots[p]);
        }
        std::vector<int> ds(deg);
        std::sort(ds.begin(), ds.end(), std::greater<int>());
        for (int j = 0; j < h.cols; ++j)
            if (ds[j] > pass_cv[j / G]) return fail(BPDC_ERR_UNSUPPORTED, "the column weights do not fit the passes");
    }
    int dc = 1;
    for (int i = 0; i < h.rows; ++i) dc = std::max(dc, h.ptr[i + 1] - h.ptr[i]);
    Layout lay;
    plan_layout(h.rows, h.cols, h.ptr, h.col, G, pv * G, dc, optimize != 0, pass_cv, lay);
    for (int j = 0; j < h.cols && !pass_cv.empty(); ++j)
        if (deg[j] > pass_cv[lay.pos_of_var[j] / G])
            return fail(BPDC_ERR_UNSUPPORTED, "the planner could not place column %d within its pass width", j);
    std::copy(lay.pos_of_var.begin(), lay.pos_of_var.end(), pos_of_var);
    // edge_round is reported in the caller's CSR order (copy_csr sorted each row)
    for (int i = 0; i < h.rows; ++i)
        for (int a = H->row_ptr[i]; a < H->row_ptr[i + 1]; ++a) {
            const int c = H->col_idx[a];
            const int b = (int)(std::lower_bound(h.col.begin() + h.ptr[i], h.col.begin() + h.ptr[i + 1], c) - h.col.begin());
            edge_round[a] = lay.edge_round[b];
        }
    return BPDC_OK;
}

int bpdc_layout_plan(const bpdc_csr *H, int32_t G, int32_t optimize, int32_t *pos_of_var, int32_t *edge_round)
{
    return bpdc_layout_plan_slots(H, G, optimize, 0, nullptr, pos_of_var, edge_round);
}

int bpdc_graph_set_layout(bpdc_graph_t g, int32_t mode)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    if (mode != 0 && mode != 1) return fail(BPDC_ERR_INVALID_ARG, "layout mode must be 0 or 1");
    const int keep = g->layout;
    g->layout = mode;
    const int rc = replan(g, 0, g->variant);
    if (rc != BPDC_OK) g->layout = keep;
    return rc;
}

int bpdc_graph_set_weights(bpdc_graph_t g, const float *weights, int32_t T, float clip)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    if (weights && (T < 1 || T > 1000)) return fail(BPDC_ERR_INVALID_ARG, "T must be in [1, 1000]");
    if (weights && (!(clip > 0.0f) || clip > 30.0f)) return fail(BPDC_ERR_INVALID_ARG, "clip must be in (0, 30]");
    if (weights && g->opts.variant != 1)
        return fail(BPDC_ERR_UNSUPPORTED, "learned weights need the product-sum check rule (variant 1)");
    const size_t E = g->H.col.size();
    std::vector<float> keep = g->w_host;
    const int keep_T = g->w_T;
    const float keep_clip = g->w_clip;
    if (weights) {
        g->w_host.assign(weights, weights + (size_t)2 * T * E);
        for (float w : g->w_host)
            if (!std::isfinite(w)) { g->w_host = keep; return fail(BPDC_ERR_INVALID_ARG, "non-finite weight"); }
        g->w_T = T;
        g->w_clip = clip;
    } else {
        g->w_host.clear();
        g->w_T = 0;
        g->w_clip = 0.0f;
    }
    const int rc = replan(g, 0, g->variant);
    if (rc != BPDC_OK) {
        g->w_host = keep;
        g->w_T = keep_T;
        g->w_clip = keep_clip;
    }
    return rc;
}

int bpdc_graph_set_kernel(bpdc_graph_t g, int32_t kernel_id)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    if (kernel_id < 0 || kernel_id >= num_variants())
        return fail(BPDC_ERR_INVALID_ARG, "kernel_id %d out of range [0, %d)", kernel_id, num_variants());
    return replan(g, 0, kernel_id);
}

int bpdc_decode(bpdc_graph_t g, int64_t B, const uint32_t *syndromes, uint64_t shot_offset,
                const bpdc_outputs *out, int persistent, void *stream)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    if (B < 0) return fail(BPDC_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return BPDC_OK;
    int rc = check_outputs(out);
    if (rc != BPDC_OK) return rc;
    if (!syndromes) return fail(BPDC_ERR_INVALID_ARG, "syndromes is NULL");
    std::lock_guard<std::mutex> lk(g->mu);
    DeviceGuard dgd(g->device);
    const int s = acquire_slot(g);
    fill_desc(g->ring[s].host_desc[0], g, B, syndromes, shot_offset, out, 0);
    return enqueue(g, s, 1, B, g->variant, g->smem_bytes, persistent != 0, (cudaStream_t)stream);
}

int bpdc_decode_multi(const bpdc_batch *batches, int32_t n, void *stream)
{
    if (n < 0 || (n > 0 && !batches)) return fail(BPDC_ERR_INVALID_ARG, "bad batch list");
    if (n == 0) return BPDC_OK;
    const int dev = batches[0].graph ? batches[0].graph->device : -1;
    for (int i = 0; i < n; ++i) {
        if (!batches[i].graph) return fail(BPDC_ERR_INVALID_ARG, "batch %d has no graph", i);
        if (batches[i].graph->device != dev) return fail(BPDC_ERR_INVALID_ARG, "graphs on different devices");
        if (batches[i].B < 0) return fail(BPDC_ERR_INVALID_ARG, "batch %d: B < 0", i);
        if (batches[i].B == 0) continue;
        if (!batches[i].syndromes) return fail(BPDC_ERR_INVALID_ARG, "batch %d: syndromes NULL", i);
        int rc = check_outputs(&batches[i].out);
        if (rc != BPDC_OK) return rc;
    }
    bpdc_graph_s *owner = batches[0].graph;
    std::lock_guard<std::mutex> lk(owner->mu);
    DeviceGuard dgd(dev);
    // one launch per kernel variant (chunks of at most kMaxBatches batches)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return batches[a].graph->variant < batches[b].graph->variant;
    });
    size_t i = 0;
    while (i < order.size()) {
        const int vid = batches[order[i]].graph->variant;
        const int s = acquire_slot(owner);
        int cnt = 0, smem = 0;
        int64_t total = 0;
        while (i < order.size() && cnt < kMaxBatches && batches[order[i]].graph->variant == vid) {
            const bpdc_batch &bt = batches[order[i]];
            // a launch takes at most kMaxLaunchShots: the next one takes the rest
            if (cnt > 0 && total + bt.B > kMaxLaunchShots) break;
            if (bt.B > 0) {
                fill_desc(owner->ring[s].host_desc[cnt], bt.graph, bt.B, bt.syndromes, bt.shot_offset, &bt.out, total);
                total += bt.B;
                smem = std::max(smem, bt.graph->smem_bytes);
                ++cnt;
            }
            ++i;
        }
        if (cnt == 0) continue;
        int rc = enqueue(owner, s, cnt, total, vid, smem, true, (cudaStream_t)stream);
        if (rc != BPDC_OK) return rc;
    }
    return BPDC_OK;
}

int bpdc_decode_host(const bpdc_batch *batches, int32_t n, int64_t chunk_shots, void *stream)
{
    if (n < 0 || (n > 0 && !batches)) return fail(BPDC_ERR_INVALID_ARG, "bad batch list");
    if (chunk_shots < 0) return fail(BPDC_ERR_INVALID_ARG, "chunk_shots < 0");
    if (n == 0) return BPDC_OK;
    const int64_t chunk = chunk_shots > 0 ? chunk_shots : kHostChunk;
    const int dev = batches[0].graph ? batches[0].graph->device : -1;
    size_t mw = 1, nw = 1, kw = 1;
    int64_t shots = 0;
    for (int i = 0; i < n; ++i) {
        const bpdc_batch &bt = batches[i];
        if (!bt.graph) return fail(BPDC_ERR_INVALID_ARG, "batch %d has no graph", i);
        if (bt.graph->device != dev) return fail(BPDC_ERR_INVALID_ARG, "graphs on different devices");
        if (bt.B < 0) return fail(BPDC_ERR_INVALID_ARG, "batch %d: B < 0", i);
        if (bt.B == 0) continue;
        if (!bt.syndromes) return fail(BPDC_ERR_INVALID_ARG, "batch %d: syndromes NULL", i);
        int rc = check_outputs(&bt.out);
        if (rc != BPDC_OK) return rc;
        if (bt.out.posterior_llr || bt.out.counters || bt.out.cut_in)
            return fail(BPDC_ERR_UNSUPPORTED,
                        "batch %d: bpdc_decode_host takes no posterior_llr, counters or cut_in", i);
        mw = std::max(mw, (size_t)bt.graph->dg.MW);
        nw = std::max(nw, (size_t)bt.graph->dg.NW);
        kw = std::max(kw, (size_t)bt.graph->dg.KW);
        shots += bt.B;
    }
    if (shots == 0) return BPDC_OK;
    // one staging set: syndromes, obs_true, corrections, logical flips,
    // iterations and status of `chunk` shots at the widest graph's row widths
    const size_t rows = (size_t)std::min<int64_t>(chunk, shots);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_syn = 0, o_obs = o_syn + al(rows * mw * 4), o_cor = o_obs + al(rows * kw * 4);
    const size_t o_lf = o_cor + al(rows * nw * 4), o_it = o_lf + al(rows * kw * 4), o_st = o_it + al(rows * 4);
    const size_t set_bytes = o_st + al(rows);

    bpdc_graph_s *owner = batches[0].graph;
    std::lock_guard<std::mutex> lk(owner->mu);
    DeviceGuard dgd(dev);
    if (!dgd.ok) return fail(BPDC_ERR_CUDA, "cannot select device %d", dev);
    cudaError_t e = cudaSuccess;
    if (!owner->copy_in) e = cudaStreamCreateWithFlags(&owner->copy_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !owner->copy_out) e = cudaStreamCreateWithFlags(&owner->copy_out, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
        if (!owner->ev_in[k]) e = cudaEventCreateWithFlags(&owner->ev_in[k], cudaEventDisableTiming);
        if (e == cudaSuccess && !owner->ev_dec[k]) e = cudaEventCreateWithFlags(&owner->ev_dec[k], cudaEventDisableTiming);
        if (e == cudaSuccess && !owner->ev_out[k]) e = cudaEventCreateWithFlags(&owner->ev_out[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && !owner->ev_entry) e = cudaEventCreateWithFlags(&owner->ev_entry, cudaEventDisableTiming);
    if (e == cudaSuccess && !owner->ev_exit) e = cudaEventCreateWithFlags(&owner->ev_exit, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "host-decode streams and events");
    if (owner->stage_set_bytes < set_bytes) {
        // every earlier call returned after its copies, so the old staging is idle
        if (owner->stage) cudaFree(owner->stage);
        owner->stage = nullptr;
        owner->stage_set_bytes = 0;
        e = lib_malloc(&owner->stage, 2 * set_bytes);
        if (e != cudaSuccess)
            return fail(BPDC_ERR_OOM, "host-decode staging of %zu bytes: %s", 2 * set_bytes, cudaGetErrorString(e));
        owner->stage_set_bytes = set_bytes;
    }
    const cudaStream_t cs = (cudaStream_t)stream;
    // the copies start after the work already queued on the caller's stream
    e = cudaEventRecord(owner->ev_entry, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(owner->copy_in, owner->ev_entry, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(owner->copy_out, owner->ev_entry, 0);
    int rc = e == cudaSuccess ? BPDC_OK : cuda_fail(e, "host-decode entry");

    // pieces of at most `chunk` shots of each batch, alternating between the
    // two staging sets: copy in (copy_in), decode (caller's stream), copy out
    // (copy_out).  The copy-in of piece k waits until the decode of piece
    // k - 2 has read its set; the decode of piece k waits for its inputs and
    // until the outputs of piece k - 2 have left the set.
    int64_t k = 0;
    for (int i = 0; i < n && rc == BPDC_OK; ++i) {
        const bpdc_batch &bt = batches[i];
        const bpdc_graph_s *g = bt.graph;
        const size_t MW = (size_t)g->dg.MW, NW = (size_t)g->dg.NW, KW = (size_t)g->dg.KW;
        for (int64_t b0 = 0; b0 < bt.B && rc == BPDC_OK; b0 += chunk, ++k) {
            const int64_t nb = std::min<int64_t>(chunk, bt.B - b0);
            const int s = (int)(k & 1);
            char *base = static_cast<char *>(owner->stage) + (size_t)s * owner->stage_set_bytes;
            uint32_t *d_syn = reinterpret_cast<uint32_t *>(base + o_syn);
            uint32_t *d_obs = reinterpret_cast<uint32_t *>(base + o_obs);
            uint32_t *d_cor = reinterpret_cast<uint32_t *>(base + o_cor);
            uint32_t *d_lf = reinterpret_cast<uint32_t *>(base + o_lf);
            uint32_t *d_it = reinterpret_cast<uint32_t *>(base + o_it);
            uint8_t *d_st = reinterpret_cast<uint8_t *>(base + o_st);
            e = cudaStreamWaitEvent(owner->copy_in, owner->ev_dec[s], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d_syn, bt.syndromes + (size_t)b0 * MW, (size_t)nb * MW * 4, cudaMemcpyDefault,
                                    owner->copy_in);
            if (e == cudaSuccess && bt.out.obs_true)
                e = cudaMemcpyAsync(d_obs, bt.out.obs_true + (size_t)b0 * KW, (size_t)nb * KW * 4,
                                    cudaMemcpyDefault, owner->copy_in);
            if (e == cudaSuccess) e = cudaEventRecord(owner->ev_in[s], owner->copy_in);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, owner->ev_in[s], 0);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, owner->ev_out[s], 0);
            if (e != cudaSuccess) { rc = cuda_fail(e, "host-decode copy-in"); break; }
            bpdc_outputs o{};
            o.corrections = d_cor;
            o.status = d_st;
            o.logical_flips = bt.out.logical_flips ? d_lf : nullptr;
            o.obs_true = bt.out.obs_true ? d_obs : nullptr;
            o.iterations = bt.out.iterations ? d_it : nullptr;
            const int slot = acquire_slot(owner);
            fill_desc(owner->ring[slot].host_desc[0], g, nb, d_syn, bt.shot_offset + (uint64_t)b0, &o, 0);
            rc = enqueue(owner, slot, 1, nb, g->variant, g->smem_bytes, true, cs);
            if (rc != BPDC_OK) break;
            e = cudaEventRecord(owner->ev_dec[s], cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(owner->copy_out, owner->ev_dec[s], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(bt.out.corrections + (size_t)b0 * NW, d_cor, (size_t)nb * NW * 4,
                                    cudaMemcpyDefault, owner->copy_out);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(bt.out.status + b0, d_st, (size_t)nb, cudaMemcpyDefault, owner->copy_out);
            if (e == cudaSuccess && bt.out.logical_flips)
                e = cudaMemcpyAsync(bt.out.logical_flips + (size_t)b0 * KW, d_lf, (size_t)nb * KW * 4,
                                    cudaMemcpyDefault, owner->copy_out);
            if (e == cudaSuccess && bt.out.iterations)
                e = cudaMemcpyAsync(bt.out.iterations + b0, d_it, (size_t)nb * 4, cudaMemcpyDefault,
                                    owner->copy_out);
            if (e == cudaSuccess) e = cudaEventRecord(owner->ev_out[s], owner->copy_out);
            if (e != cudaSuccess) rc = cuda_fail(e, "host-decode copy-out");
        }
    }
    // synchronous: every copy has landed when the call returns (also after an
    // error, so that no copy into the caller's buffers is still in flight);
    // the caller's stream is left ordered after the last copy-out
    cudaError_t e1 = cudaEventRecord(owner->ev_exit, owner->copy_out);
    if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(cs, owner->ev_exit, 0);
    const cudaError_t e2 = cudaStreamSynchronize(owner->copy_in);
    const cudaError_t e3 = cudaStreamSynchronize(owner->copy_out);
    const cudaError_t e4 = cudaStreamSynchronize(cs);
    if (rc != BPDC_OK) return rc;
    for (cudaError_t x : {e1, e2, e3, e4})
        if (x != cudaSuccess) return cuda_fail(x, "host-decode completion");
    return BPDC_OK;
}

int bpdc_decode_multi_noalloc(const bpdc_batch *batches, int32_t n, void *stream)
{
    if (n < 0 || (n > 0 && !batches)) return fail(BPDC_ERR_INVALID_ARG, "bad batch list");
    if (n == 0) return BPDC_OK;
    if (n > kStaticBatches)
        return fail(BPDC_ERR_UNSUPPORTED, "bpdc_decode_multi_noalloc takes at most %d batches per call (got %d)",
                    kStaticBatches, n);
    const int dev = batches[0].graph ? batches[0].graph->device : -1;
    int vid = -1;
    for (int i = 0; i < n; ++i) {
        if (!batches[i].graph) return fail(BPDC_ERR_INVALID_ARG, "batch %d has no graph", i);
        if (batches[i].graph->device != dev) return fail(BPDC_ERR_INVALID_ARG, "graphs on different devices");
        if (batches[i].B < 0) return fail(BPDC_ERR_INVALID_ARG, "batch %d: B < 0", i);
        if (vid < 0) vid = batches[i].graph->variant;
        if (batches[i].graph->variant != vid)
            return fail(BPDC_ERR_UNSUPPORTED, "bpdc_decode_multi_noalloc needs every graph on one kernel variant");
        if (batches[i].B == 0) continue;
        if (!batches[i].syndromes) return fail(BPDC_ERR_INVALID_ARG, "batch %d: syndromes NULL", i);
        int rc = check_outputs(&batches[i].out);
        if (rc != BPDC_OK) return rc;
    }
    bpdc_graph_s *owner = batches[0].graph;
    std::lock_guard<std::mutex> lk(owner->mu);
    DeviceGuard dgd(dev);
    if (!dgd.ok) return fail(BPDC_ERR_CUDA, "cannot select device %d", dev);
    BatchDesc descs[kStaticBatches];   // host stack: no allocation
    int cnt = 0, smem = 0, bps = 0;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const bpdc_batch &bt = batches[i];
        if (bt.B == 0) continue;
        fill_desc(descs[cnt], bt.graph, bt.B, bt.syndromes, bt.shot_offset, &bt.out, total);
        total += bt.B;
        if (bt.graph->smem_bytes >= smem) {
            smem = bt.graph->smem_bytes;
            bps = bt.graph->blocks_per_sm;
        }
        ++cnt;
    }
    if (cnt == 0) return BPDC_OK;
    if (total > kMaxLaunchShots)
        return fail(BPDC_ERR_UNSUPPORTED, "at most %lld shots per call (got %lld)", (long long)kMaxLaunchShots,
                    (long long)total);
    const Variant &v = variant(vid);
    const int64_t need = (total + v.block_threads / v.G - 1) / (v.block_threads / v.G);
    const int64_t grid = std::min<int64_t>((int64_t)owner->sm_count * bps, need);
    cudaError_t e = launch_variant_static(vid, descs, cnt, total, (int)grid, smem, (cudaStream_t)stream);
    return e == cudaSuccess ? BPDC_OK : cuda_fail(e, "allocation-free decode launch");
}

int bpdc_cut_select(bpdc_graph_t g, int64_t B, const float *posterior_llr, uint64_t shot_offset,
                    uint32_t *cut_out, void *stream)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    if (B < 0) return fail(BPDC_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return BPDC_OK;
    if (!posterior_llr || !cut_out) return fail(BPDC_ERR_INVALID_ARG, "NULL buffer");
    DeviceGuard dgd(g->device);
    cudaError_t e = launch_cut_select(g->dg, B, posterior_llr, shot_offset, cut_out, (cudaStream_t)stream);
    return e == cudaSuccess ? BPDC_OK : cuda_fail(e, "cut-select launch");
}

int bpdc_sample(bpdc_graph_t g, int64_t B, uint64_t seed, uint64_t shot_offset, uint32_t *syndromes,
                uint32_t *observables, uint32_t *errors, void *stream)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    if (B < 0) return fail(BPDC_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return BPDC_OK;
    if (!syndromes) return fail(BPDC_ERR_INVALID_ARG, "syndromes is NULL");
    DeviceGuard dgd(g->device);
    cudaError_t e = launch_sample(g->dg, B, seed, shot_offset, syndromes, observables, errors, (cudaStream_t)stream);
    return e == cudaSuccess ? BPDC_OK : cuda_fail(e, "sampler launch");
}

int bpdc_graph_sync_status(bpdc_graph_t g, void *stream)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    DeviceGuard dgd(g->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    int32_t flag = 0;
    e = cudaMemcpy(&flag, g->dg.err_flag, sizeof(flag), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (flag != 0) {
        const int32_t zero = 0;
        cudaMemcpy(g->dg.err_flag, &zero, sizeof(zero), cudaMemcpyHostToDevice);
        return fail(flag, "device reported error %d", flag);
    }
    return BPDC_OK;
}

int bpdc_debug_fail_allocations(int32_t skip, int32_t count)
{
    if (skip < 0 || count < 0) return fail(BPDC_ERR_INVALID_ARG, "skip and count must be >= 0");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc_skip = count > 0 ? skip : 0;
    g_alloc_fail = count;
    return BPDC_OK;
}

int bpdc_check_status(int32_t device, int32_t *site, int64_t *index)
{
    if (!site || !index) return fail(BPDC_ERR_INVALID_ARG, "bpdc_check_status: NULL output");
#ifndef BPDC_CHECKS
    (void)device;
    return fail(BPDC_ERR_UNSUPPORTED, "bounds checks are compiled only into libbpdc_checked.so");
#else
    DeviceGuard dgd(device);
    if (!dgd.ok) return fail(BPDC_ERR_CUDA, "cannot select device %d", device);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "device synchronize");
    int s = 0;
    long long i = 0;
    if (!check_status(&s, &i)) return fail(BPDC_ERR_CUDA, "bounds-check latch unreadable");
    *site = s;
    *index = (int64_t)i;
    if (s != 0) return fail(BPDC_ERR_CHECK, "bounds check failed at site %d, index %lld", s, i);
    return BPDC_OK;
#endif
}

int bpdc_measure_smem_peak(int32_t device, int32_t reps, double *bytes_per_second, int32_t *num_sms)
{
    if (!bytes_per_second || !num_sms || reps < 8)
        return fail(BPDC_ERR_INVALID_ARG, "bpdc_measure_smem_peak: NULL output or reps < 8");
    DeviceGuard dgd(device);
    if (!dgd.ok) return fail(BPDC_ERR_CUDA, "cannot select device %d", device);
    int sms = 0;
    cudaError_t e = measure_smem_peak(reps, bytes_per_second, &sms);
    if (e != cudaSuccess) return cuda_fail(e, "shared-memory microbenchmark");
    *num_sms = sms;
    return BPDC_OK;
}

// Shared checks of the weighted-BP calls; fills the kernel arguments.
static int wbp_prepare(bpdc_graph_t g, int64_t B, const uint32_t *syndromes, const float *weights, int32_t T,
                       float clip, int32_t ckpt_every, void *workspace, size_t workspace_bytes, WbpArgs &a)
{
    if (!g) return fail(BPDC_ERR_INVALID_ARG, "graph is NULL");
    if (B < 0) return fail(BPDC_ERR_INVALID_ARG, "B < 0");
    if (T < 1 || T > 1000) return fail(BPDC_ERR_INVALID_ARG, "T must be in [1, 1000]");
    if (ckpt_every < 1 || ckpt_every > T) return fail(BPDC_ERR_INVALID_ARG, "ckpt_every must be in [1, T]");
    if (!(clip > 0.0f) || clip > 30.0f) return fail(BPDC_ERR_INVALID_ARG, "clip must be in (0, 30]");
    if (B > 0 && (!syndromes || !weights)) return fail(BPDC_ERR_INVALID_ARG, "NULL syndromes or weights");
    int rmin = 1 << 30, rmax = 0, cmax = 0;
    std::vector<int> deg(g->H.cols, 0);
    for (int i = 0; i < g->H.rows; ++i) {
        const int d = g->H.ptr[i + 1] - g->H.ptr[i];
        rmin = std::min(rmin, d);
        rmax = std::max(rmax, d);
    }
    for (int32_t c : g->H.col) cmax = std::max(cmax, ++deg[c]);
    if (rmin < 2 || rmax > kWbpMaxRow || cmax > kWbpMaxCol)
        return fail(BPDC_ERR_UNSUPPORTED, "weighted BP needs row weights in [2, %d] and column weights <= %d",
                    kWbpMaxRow, kWbpMaxCol);
    const int E = (int)g->H.col.size();
    if (wbp_smem_backward(E, ckpt_every, 1) > kMaxWbpSmem)
        return fail(BPDC_ERR_UNSUPPORTED, "graph too large for the weighted-BP adjoint (%d edges)", E);
    size_t need = 0;
    bpdc_wbp_workspace_size(g, B, T, ckpt_every, &need);
    if (B > 0 && (!workspace || workspace_bytes < need))
        return fail(BPDC_ERR_INVALID_ARG, "workspace of %zu bytes needed", need);
    const size_t nck = (size_t)B * ((T + ckpt_every - 1) / ckpt_every) * E;
    a = WbpArgs{};
    a.B = B; a.E = E; a.T = T; a.k = ckpt_every; a.clip = clip;
    a.syn = syndromes; a.W = weights;
    a.ckpt = (float *)workspace;
    a.part = (float *)workspace + ((nck + 63) & ~(size_t)63);
    return BPDC_OK;
}

int bpdc_wbp_workspace_size(bpdc_graph_t g, int64_t B, int32_t T, int32_t ckpt_every, size_t *bytes)
{
    if (!g || !bytes || B < 0 || T < 1 || ckpt_every < 1)
        return fail(BPDC_ERR_INVALID_ARG, "bpdc_wbp_workspace_size: bad argument");
    const size_t E = g->H.col.size();
    const size_t nck = (size_t)B * ((T + ckpt_every - 1) / ckpt_every) * E;
    *bytes = (((nck + 63) & ~(size_t)63) + (size_t)B * 2 * T * E) * sizeof(float);
    return BPDC_OK;
}

int bpdc_wbp_forward(bpdc_graph_t g, int64_t B, const uint32_t *syndromes, const float *weights, int32_t T,
                     float clip, int32_t ckpt_every, float *posteriors, void *workspace, size_t workspace_bytes,
                     void *stream)
{
    WbpArgs a;
    int rc = wbp_prepare(g, B, syndromes, weights, T, clip, ckpt_every, workspace, workspace_bytes, a);
    if (rc != BPDC_OK || B == 0) return rc;
    a.post = posteriors;
    DeviceGuard dgd(g->device);
    cudaError_t e = launch_wbp_forward(g->dg, a, (cudaStream_t)stream);
    return e == cudaSuccess ? BPDC_OK : cuda_fail(e, "weighted-BP forward launch");
}

int bpdc_decode_backward(bpdc_graph_t g, int64_t B, const uint32_t *syndromes, const float *weights, int32_t T,
                         float clip, int32_t ckpt_every, const float *grad_posteriors, float *grad_weights,
                         void *workspace, size_t workspace_bytes, void *stream)
{
    WbpArgs a;
    int rc = wbp_prepare(g, B, syndromes, weights, T, clip, ckpt_every, workspace, workspace_bytes, a);
    if (rc != BPDC_OK) return rc;
    if (!grad_weights || (B > 0 && !grad_posteriors))
        return fail(BPDC_ERR_INVALID_ARG, "NULL gradient buffer");
    a.gpost = grad_posteriors;
    DeviceGuard dgd(g->device);
    cudaError_t e = launch_wbp_backward(g->dg, a, grad_weights, (cudaStream_t)stream);
    return e == cudaSuccess ? BPDC_OK : cuda_fail(e, "weighted-BP backward launch");
}

}  // extern "C"
