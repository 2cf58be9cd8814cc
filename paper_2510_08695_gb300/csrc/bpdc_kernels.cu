// BP+DC decoding kernels for sm_103a (arXiv 2510.08695, Sec. II.C.1 and
// Algorithms 1-2).
//
// Mapping: a group of G threads decodes one shot at a time.  The shot's
// message state lives in shared memory as one FP32 slot per Tanner-graph
// edge, arranged variable-major (slot(p, m, u) = (p*cv + m)*G + u for the
// m-th edge of the variable at lane u, pass p), so the variable update reads
// and writes consecutive words across lanes.  The check update gathers the
// slots of its row through per-lane slot indices kept in registers and
// scatters its answers back into the same slots: every slot alternates
// between the variable->check message q (after the variable update) and the
// check->variable message r (after the check update).
//
// Flooding iteration t (t = 1 .. T_iter + 1):
//   check phase   for every check: gather q of its row, test the row parity of
//                 the current hard decision (carried in the least significant
//                 mantissa bit of each q, see below), form sign / min1 / min2
//                 and, if t <= T_iter, scatter r = alpha * sign * min(others).
//   reduce        group-wide OR of the row-parity mismatches (a barrier that
//                 also publishes the scatter).  None left: the hard decision
//                 of iteration t-1 reproduces the syndrome -> converged after
//                 t-1 iterations.  t = T_iter + 1: failed.
//   variable      posterior L = lambda + sum r, hard decision e = [L <= 0]
//   phase         (Eq. 4), extrinsic q = lambda + sum of the other r, tagged
//                 with e; at t = T_iter slot 0 keeps the tagged L instead of q
//                 so that the cut selection can read it.
//
// Tag: the variable update stores e_j in the least significant mantissa bit
// of every q it writes (a change of at most one unit in the last place,
// 2^-23 relative), so the check phase obtains the parity of the hard
// decision over its row by XOR-ing the words it already loads.  Cut
// variables send q = +inf (tag 0, e = 0): they never win a minimum, add no
// sign and no parity, which is the column deletion of Algorithm 1 and the
// zero prior of Algorithm 2.  Denormals must not be flushed (no -ftz).
//
// Degeneracy cutting (the selection step of Algorithm 1): on failure every row of D
// gathers the tagged L^T of its support from slot 0, takes the windowed
// maximum, breaks ties with the SplitMix64 hash of (shot, row) and sets the
// winner's bit in a shared cut mask; BP runs again with cut variables pinned
// to +inf and the priors of Sec. III.B.
#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <cuda_runtime.h>

#include "bpdc_internal.h"

namespace bpdc {
namespace {
#ifdef BPDC_CHECKS
// Checked build (libbpdc_checked.so): the first failed bounds check on the
// device latches (site, index) here and the access is skipped; nothing traps.
__device__ unsigned long long g_check[2];

__device__ __forceinline__ void check_fail(int site, long long idx)
{
    if (atomicCAS(&g_check[0], 0ull, (unsigned long long)site) == 0ull) atomicExch(&g_check[1], (unsigned long long)idx);
}

__device__ __forceinline__ bool check_index(int site, long long idx, long long len)
{
    if (idx >= 0 && idx < len) return true;
    check_fail(site, idx);
    return false;
}

// a 4-byte access at shared address a lies inside the block's dynamic shared
// memory and is aligned
__device__ __forceinline__ bool smem_ok(uint32_t a, int site)
{
    extern __shared__ uint32_t smem_all[];
    const uint32_t lo = (uint32_t)__cvta_generic_to_shared(smem_all);
    uint32_t size;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
    if (a >= lo && a + 4u <= lo + size && (a & 3u) == 0u) return true;
    check_fail(site, (long long)a - (long long)lo);
    return false;
}

// the position j has a column and the column indexes a posterior row
__device__ __forceinline__ bool post_ok(const DevGraph &g, long long j)
{
    return check_index(5, j, g.n_pos) && check_index(7, __ldg(g.pos_col + j), g.N);
}
#endif


__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

// SplitMix64 output number ctr of the stream keyed by key (Steele, Lea &
// Flood 2014).
__device__ __forceinline__ uint64_t splitmix64(uint64_t key, uint64_t ctr)
{
    uint64_t z = key + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Synchronisation of the G threads that share a shot.
template <int G>
struct Group {
    int u;          // lane within the group
    int bar;        // named barrier id (G > 32)
    unsigned mask;  // lanes of the warp that belong to the group (G <= 32)
    int leader;     // warp lane of the group's lane 0 (G <= 32)

    __device__ __forceinline__ void sync() const
    {
        if constexpr (G <= 32) {
            __syncwarp(mask);
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(G) : "memory");
        }
    }
    // Barrier that also returns whether any lane passed a true predicate.
    __device__ __forceinline__ bool any(bool p) const
    {
        if constexpr (G <= 32) {
            __syncwarp(mask);
            return __any_sync(mask, p) != 0;
        } else {
            uint32_t r;
            asm volatile(
                "{\n\t.reg .pred pi, po;\n\t"
                "setp.ne.u32 pi, %1, 0;\n\t"
                "bar.red.or.pred po, %2, %3, pi;\n\t"
                "selp.u32 %0, 1, 0, po;\n\t}"
                : "=r"(r)
                : "r"((uint32_t)p), "r"(bar), "n"(G)
                : "memory");
            return r != 0;
        }
    }
};

// The cut of Algorithm 1 for one shot: every row of D picks the
// support variable of largest posterior LLR (windowed, hashed tie-break;
// candidates in ascending column order) and marks it.  load(a, e) returns the
// posterior of D entry a (e = its packed slot | position word); mark(a, e)
// records the winner.
template <typename LoadL, typename Mark>
__device__ __forceinline__ void cut_rows(const DevGraph &g, uint64_t gshot, int u, int G, LoadL load,
                                         Mark mark)
{
    for (int r = u; r < g.Md; r += G) {
        const int b0 = __ldg(g.d_ptr + r), b1 = __ldg(g.d_ptr + r + 1);
#ifdef BPDC_CHECKS
        if (b0 < b1 && (!check_index(6, b0, g.n_d_ent) || !check_index(6, b1 - 1, g.n_d_ent))) continue;
#endif
        if (b0 == b1) continue;
        float lmax = -f_inf();
        for (int a = b0; a < b1; ++a) {
            const uint32_t e = __ldg(g.d_ent + a);
            lmax = fmaxf(lmax, load(a, e));
        }
        const float thr = isfinite(lmax) ? lmax - g.tie_rel * fmaxf(1.0f, fabsf(lmax)) : lmax;
        int nc = 0;
        for (int a = b0; a < b1; ++a) {
            const uint32_t e = __ldg(g.d_ent + a);
            nc += load(a, e) >= thr;
        }
        if (nc == 0) continue;   // only with NaN posteriors
        const uint64_t h = splitmix64(g.tie_seed, gshot * (uint64_t)g.Md + (uint64_t)r);
        int pick = (int)(h % (uint64_t)nc);
        for (int a = b0; a < b1; ++a) {
            const uint32_t e = __ldg(g.d_ent + a);
            if (load(a, e) >= thr) {
                if (pick == 0) { mark(a, e); break; }
                --pick;
            }
        }
    }
}

// phi(x) = -log(tanh(x / 2)) for x >= 0 (phi(0) = +inf, phi(+inf) = 0); phi is
// its own inverse and 2 atanh(prod tanh(x_j / 2)) = phi(sum phi(x_j)), the
// product-sum check rule (Sec. II.C.1 cites it) in a form that keeps FP32
// accurate: expm1 and log1p avoid the cancellations of tanh near 1.
__device__ __forceinline__ float phi(float x) { return log1pf(2.0f / expm1f(x)); }

// phi(x) = 2 atanh(e^-x) falls below the smallest normal FP32 number once
// x > ~87, so a sum of phi terms whose smallest argument m is large would
// vanish and its phi would come out +inf.  Sums are therefore taken with every
// argument lowered by s = max(0, m - kPhiShift): where s > 0 every argument is
// >= kPhiShift, phi(x) = 2 e^-x to within a relative e^-2x, and
// phi(sum_j phi(x_j)) = -log sum_j e^-x_j + O(e^-2m), which lowers by exactly s.
constexpr float kPhiShift = 20.0f;

// A check's minimum |q| as it enters the outgoing message, scaled by a (the
// min-sum scale, or 1): at most the cap, and 0 below the smallest normal
// float.  The hard-decision tag turns a message that is exactly 0 into the
// smallest denormal when its sender's decision is 1; without the flush that
// denormal would move an exact 0 of the rule (and with it a posterior L = 0,
// whose decision is 1) off zero.  The multiply flushes a denormal operand (and
// result) to zero itself (.ftz), so the flush costs no instruction; no
// message of the rule is nonzero and that small otherwise.
__device__ __forceinline__ float scaled_min(float a, float m)
{
    float r;
    asm("mul.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(fminf(m, kLlrCap)));
    return r;
}

// Shared words at the start of every group's region: 0-1 shot broadcast
// (double buffered), 2 the +inf word, 4-11 the per-batch counters.
constexpr int kMiscWords = 12;

__device__ __forceinline__ uint32_t lds32(uint32_t a)
{
#ifdef BPDC_CHECKS
    if (!smem_ok(a, 1)) return 0u;
#endif
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// The same load typed as a float, so that |x| folds into the compare and
// min / max instructions as an operand modifier instead of a separate mask.
__device__ __forceinline__ float ldsf(uint32_t a)
{
#ifdef BPDC_CHECKS
    if (!smem_ok(a, 1)) return 0.0f;
#endif
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

// Minimum of three floats in one instruction (sm_100 and later).
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// 16-byte load of a table entry (four words).
__device__ __forceinline__ uint4 lds128(uint32_t a)
{
#ifdef BPDC_CHECKS
    if (!smem_ok(a, 1) || !smem_ok(a + 12u, 1)) return make_uint4(0x20002u, 0x20002u, 0x20002u, 0x20002u);
#endif
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts32(uint32_t a, uint32_t v)
{
#ifdef BPDC_CHECKS
    if (!smem_ok(a, 2)) return;
#endif
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(a), "r"(v));
}

// Store under a predicate evaluated inside the PTX, so that the compiler
// emits one predicated store instead of a branch around the inline asm.
__device__ __forceinline__ void sts32_if(uint32_t a, uint32_t v, bool pred)
{
#ifdef BPDC_CHECKS
    if (pred && !smem_ok(a, 2)) return;
#endif
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.u32 q, %2, 0;\n\t"
        "@q st.shared.b32 [%0], %1;\n\t}" ::"r"(a), "r"(v), "r"((uint32_t)pred));
}

// Per-lane state that depends only on the graph (reloaded when a launch
// switches to a batch of another graph).  CMIN: every variable has at least
// CMIN edges (slots below CMIN need no store predicate); RC: every check has
// exactly DCM edges.
template <int G, int PCM, int DCM, int PVM, int CVM, int CMIN, bool RC, uint64_t PROF, bool TAB>
struct Lane {
    // slots of pass p (per lane) and the slots before it
    static constexpr int cv(int p) { return prof_cv(PROF, CVM, p); }
    static constexpr int off(int p) { return prof_off(PROF, CVM, p); }
    static constexpr int kSlotsPerLane = prof_off(PROF, CVM, PVM);
    static constexpr int kVmWords = (kSlotsPerLane + 31) / 32;

    static constexpr bool kWide = wide_slots(G, kSlotsPerLane);
    // wide form with the check-edge word indices in shared memory: 16-byte
    // entries of 8 indices, entry c of pass p of this lane at
    // tab + 16 * (p * kTabChunks + c) * G
    static constexpr bool kTab = kWide && TAB;
    static constexpr int kTabChunks = (DCM + kTabEdges - 1) / kTabEdges;
    static_assert(!kTab || kTabChunks > 0, "a shared edge table needs rows");
    // rows longer than 16 keep the gathered q in registers for the scatter
    // when a thread has the registers for it (512 threads or fewer per SM);
    // else the scatter reads each q again
    static constexpr bool kHoldLong = kTab && G <= 512;
    static_assert(!kHoldLong || kTab, "held long rows need the shared edge table");

    __device__ __forceinline__ uint32_t tab_entry(int p, int c) const
    {
        return tab + 16u * G * (uint32_t)(p * kTabChunks + c);
    }
    // shared byte address of each check edge's slot (the +inf word if none):
    // one register per edge when a lane has at most 40 check edges (no
    // unpacking at each access), else two 16-bit values per register.  The
    // wide form (a group larger than 64 KB, one per SM, 64 registers per
    // thread) keeps none: it reads the word index of the edge from the
    // read-only table chk_word at each access (coalesced 2-byte loads), so
    // that its registers do not spill.
    static constexpr bool kFullAddr = !kWide && PCM * DCM <= 40;
    static constexpr int kAddrWords = kWide ? 1 : kFullAddr ? PCM * DCM : (PCM * DCM + 1) / 2;
    uint32_t aw[kAddrWords];
    const uint16_t *cw;        // wide form: this lane's column of chk_word ([pc][DCM][G])
    uint32_t tab;              // wide form with a table: shared byte address of this lane's entry 0
#ifdef BPDC_CHECKS
    const uint16_t *cw0;       // chk_word and its length (checked build)
    long long n_cw;
#endif
    uint32_t region_base;      // shared byte address of the group's region (wide form)
    uint32_t slot_base;        // shared byte address of slot 0
    uint32_t vm[kVmWords];     // bit (p*CVM + m): the variable at pass p has an m-th edge
    uint32_t vvalid;           // bit p: a variable sits at pass p
    uint32_t cvalid;           // bit p: a check sits at pass p
    float lamv[PVM];           // prior LLR per variable pass (+inf past N)
    uint32_t lane_base;        // shared byte address of slot(0, 0, u)
    uint32_t inf_addr;         // shared byte address of the group's +inf word

    __device__ __forceinline__ bool has(int p, int m) const
    {
        const int n = off(p) + m;
        return (vm[n >> 5] >> (n & 31)) & 1u;
    }

    // Shared byte address of the word with index w of the group's region.
    __device__ __forceinline__ uint32_t word_addr(uint32_t w) const { return region_base + 4u * w; }

    __device__ __forceinline__ uint32_t addr(int p, int k) const
    {
        if constexpr (kWide) {
#ifdef BPDC_CHECKS
            if (!check_index(4, (long long)(cw - cw0) + (long long)(p * DCM + k) * G, n_cw)) return inf_addr;
#endif
            return region_base + 4u * (uint32_t)__ldg(cw + (p * DCM + k) * G);
        } else {
            const int n = p * DCM + k;
            if constexpr (kFullAddr) return aw[n];
            else return (n & 1) ? (aw[n >> 1] >> 16) : (aw[n >> 1] & 0xFFFFu);
        }
    }

    __device__ void reload_lam(const DevGraph &g, int u)
    {
#pragma unroll
        for (int p = 0; p < PVM; ++p) {
            const int j = p * G + u;
            (void)j;
#ifdef BPDC_CHECKS
            if (p < g.pv && !check_index(5, (long long)p * G + u, g.n_pos)) { lamv[p] = f_inf(); continue; }
#endif
            lamv[p] = p < g.pv ? __ldg(g.lam + (size_t)p * G + u) : f_inf();
        }
    }

    __device__ void load(const DevGraph &g, int u, uint32_t slot_base, uint32_t inf_word)
    {
        lane_base = slot_base + 4u * (uint32_t)u;
        inf_addr = inf_word;
        region_base = slot_base - 4u * kMiscWords;
        this->slot_base = slot_base;
        cvalid = 0;
        cw = g.chk_word + u;
        tab = region_base + 4u * (uint32_t)g.tab_off + 16u * (uint32_t)u;
        if constexpr (kTab) {
            // this lane's entries of the edge table into shared memory; only
            // this lane reads them back, so no barrier is needed
#pragma unroll
            for (int p = 0; p < PCM; ++p) {
                if (p >= g.pc) break;
#pragma unroll
                for (int c = 0; c < kTabChunks; ++c) {
                    const uint4 e = __ldg(g.chk_tab + ((size_t)p * kTabChunks + c) * G + u);
                    const uint32_t a = tab_entry(p, c);
#ifdef BPDC_CHECKS
                    if (!smem_ok(a, 2) || !smem_ok(a + 12u, 2)) continue;
#endif
                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(e.x), "r"(e.y), "r"(e.z),
                                 "r"(e.w));
                }
            }
        }
#ifdef BPDC_CHECKS
        cw0 = g.chk_word;
        n_cw = g.n_chk_word;
#endif
#pragma unroll
        for (int w = 0; w < kAddrWords; ++w) aw[w] = 0;
#pragma unroll
        for (int p = 0; p < PCM; ++p) {
            if (p < g.pc && p * G + u < g.M) cvalid |= 1u << p;
            if constexpr (!kWide) {
#pragma unroll
                for (int k = 0; k < DCM; ++k) {
                    uint32_t v = kNoEdge;
#ifdef BPDC_CHECKS
                    if (p < g.pc && k < g.dc && !check_index(3, ((long long)p * g.dc + k) * G + u, g.n_chk_idx)) {} else
#endif
                    if (p < g.pc && k < g.dc) v = __ldg(g.chk_idx + ((size_t)p * g.dc + k) * G + u);
                    const uint32_t a = ((v == kNoEdge) ? inf_word : slot_base + 4u * v) & 0xFFFFu;
                    const int n = p * DCM + k;
                    if constexpr (kFullAddr) aw[n] = a;
                    else aw[n >> 1] |= a << ((n & 1) * 16);
                }
            }
        }
#pragma unroll
        for (int w = 0; w < kVmWords; ++w) vm[w] = 0;
        vvalid = 0;
#pragma unroll
        for (int p = 0; p < PVM; ++p) {
            const int j = p * G + u;
            int deg = 0;
            (void)j;
            if (p < g.pv) {
#ifdef BPDC_CHECKS
                if (!check_index(5, (long long)p * G + u, g.n_pos)) continue;
#endif
                deg = __ldg(g.var_deg + (size_t)p * G + u);
                if (deg == 0xFF) deg = 0; else vvalid |= 1u << p;
            }
#pragma unroll
            for (int m = 0; m < CVM; ++m) {
                const int n = off(p) + m;
                if (m < cv(p) && m < deg) vm[n >> 5] |= 1u << (n & 31);
            }
        }
        reload_lam(g, u);
    }
};

// TAIL > 0 (one warp per shot): the last check pass holds up to 32 / TAIL
// checks, each spread over TAIL consecutive lanes (see tail_pass).
template <int G, int PCM, int DCM, int PVM, int CVM, int CMIN, bool RC, int RULE, uint64_t PROF, bool TAB,
          int TAIL>
struct Decoder {
    using L = Lane<G, PCM, DCM, PVM, CVM, CMIN, RC, PROF, TAB>;
    static constexpr uint32_t kSlot = 4u * G;         // bytes between a variable's slots
    static_assert(TAIL == 0 || (G == 32 && RULE == 0 && (TAIL & (TAIL - 1)) == 0 && TAIL <= 32),
                  "a shared last check pass needs one warp per shot, min-sum and a power-of-two lane count");

    // shared byte address of slot 0 of this lane's variable at pass p
    static __device__ __forceinline__ uint32_t pass_base(const L &ln, int p)
    {
        return ln.lane_base + 4u * G * (uint32_t)L::off(p);
    }

    // The last check pass of a variant with TAIL > 0: check c of the pass sits
    // on lanes c*TAIL .. c*TAIL+TAIL-1, and each of those lanes holds
    // kTailEdges of its edges (the +inf word where the check has fewer).  Every
    // lane takes the two smallest |q| and the sign / hard-decision parity of
    // its own edges, the lanes of a check combine theirs by butterfly
    // shuffles (the smallest two of a union are min(a1, b1) and
    // min(max(a1, b1), a2, b2): exact, in any order), and each lane then
    // answers its own edges as the one-lane update would.  Only the check's
    // first lane carries the syndrome bit.  A short last pass (a few checks
    // past a multiple of 32) thus costs about a lane's share of a full one.
    // Returns the check's parity word (bit 0: unsatisfied).
    static __device__ __forceinline__ uint32_t tail_pass(const L &ln, int p, uint32_t sbits, float alpha,
                                                         bool scatter)
    {
        constexpr int E = (DCM + TAIL - 1) / (TAIL > 0 ? TAIL : 1);   // edges per lane
        uint32_t S = ((sbits >> p) & 1u) * 0x80000001u;
        float mn1 = f_inf(), mn2 = f_inf();
        float qf[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const float v = ldsf(ln.addr(p, k));
            qf[k] = v;
            S ^= __float_as_uint(v);
            const float av = fabsf(v);
            mn2 = fminf(mn2, fmaxf(mn1, av));
            mn1 = fminf(mn1, av);
        }
#pragma unroll
        for (int o = TAIL / 2; o >= 1; o >>= 1) {
            const float o1 = __shfl_xor_sync(0xFFFFFFFFu, mn1, o);
            const float o2 = __shfl_xor_sync(0xFFFFFFFFu, mn2, o);
            S ^= __shfl_xor_sync(0xFFFFFFFFu, S, o);
            mn2 = fmin3(fmaxf(mn1, o1), mn2, o2);
            mn1 = fminf(mn1, o1);
        }
        if (scatter) {
            const float sa = __uint_as_float(__float_as_uint(alpha) ^ (S & 0x80000000u));
            const uint32_t m1 = __float_as_uint(scaled_min(sa, mn1));
            const uint32_t m2 = __float_as_uint(scaled_min(sa, mn2));
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const uint32_t a = ln.addr(p, k);
                const bool is_min = fabsf(qf[k]) == mn1;
                sts32_if(a, (is_min ? m2 : m1) ^ (__float_as_uint(qf[k]) & 0x80000000u), a != ln.inf_addr);
            }
        }
        return S;
    }

    // Initial messages of a BP run: every variable announces its prior LLR
    // tagged with its hard decision (cut variables carry lambda = +inf);
    // unused slots are zero.  Returns the hard-decision bits per pass.
    static __device__ __forceinline__ uint32_t init(const DevGraph &g, const L &ln, int u, float *post_row)
    {
        uint32_t hd = 0;
#pragma unroll
        for (int p = 0; p < PVM; ++p) {
            if (p < g.pv) {
                const float lam = ln.lamv[p];
                const uint32_t e = lam <= 0.0f ? 1u : 0u;
                hd |= e << p;
                const uint32_t v = (__float_as_uint(lam) & ~1u) | e;
                const uint32_t base = pass_base(ln, p);
                if (RULE == 1 && g.wts) {   // weighted BP: q = clip(wv[0] lambda) per edge
                    const float *wv = g.wts + (size_t)g.w_T * g.slots;
#pragma unroll
                    for (int m = 0; m < CVM; ++m) {
                        if (m >= L::cv(p)) continue;
                        const bool on = m < CMIN || ln.has(p, m);
                        const float q = on ? fminf(fmaxf(__ldg(wv + (L::off(p) + m) * G + u) * lam, -g.w_clip), g.w_clip)
                                           : 0.0f;
                        sts32(base + m * kSlot, on ? ((__float_as_uint(q) & ~1u) | e) : 0u);
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < CVM; ++m)
                        if (m < L::cv(p)) sts32(base + m * kSlot, (m < CMIN || ln.has(p, m)) ? v : 0u);
                }
#ifdef BPDC_CHECKS
                if (post_row && ((ln.vvalid >> p) & 1u) && !post_ok(g, (long long)p * G + u)) {} else
#endif
                if (post_row && ((ln.vvalid >> p) & 1u)) post_row[__ldg(g.pos_col + p * G + u)] = lam;
            }
        }
        return hd & ln.vvalid;
    }

    // Variable update at pass P (CVP = L::cv(P) slots per variable): the
    // posterior L = lambda + sum r, the hard decision e = [L <= 0] (Eq. 4) and
    // the extrinsic messages q = lambda + the other r (prefix and suffix
    // sums), stored tagged with e; at the last iteration slot 0 keeps the
    // tagged L for the cut selection.  Slots past a variable's degree hold 0,
    // so a pass wider than the degree adds exact zeros.  Returns e.
    template <bool FAST, int P>
    static __device__ __forceinline__ uint32_t var_pass(const DevGraph &g, const L &ln, int u, int t, bool last,
                                                        float *post_row)
    {
        constexpr int CVP = L::cv(P);
        const uint32_t base = pass_base(ln, P);
        float r[CVP];
#pragma unroll
        for (int m = 0; m < CVP; ++m) r[m] = __uint_as_float(lds32(base + m * kSlot));
        float pre[CVP + 1];
        pre[0] = ln.lamv[P];
#pragma unroll
        for (int m = 0; m < CVP; ++m) pre[m + 1] = pre[m] + r[m];
        float suf[CVP + 1];
        suf[CVP] = 0.0f;
        suf[CVP - 1] = r[CVP - 1];
#pragma unroll
        for (int m = CVP - 2; m >= 1; --m) suf[m] = r[m] + suf[m + 1];
        const float Lp = pre[CVP];
        const uint32_t e = Lp <= 0.0f ? 1u : 0u;
        const float *wv = (RULE == 1 && g.wts)
            ? g.wts + ((size_t)g.w_T + min(t + 1, g.w_T) - 1) * g.slots + L::off(P) * G + u
            : nullptr;
#pragma unroll
        for (int m = 0; m < CVP; ++m) {
            float q = (m == CVP - 1) ? pre[m] : pre[m] + suf[m + 1];
            if (RULE == 1 && wv) q = fminf(fmaxf(__ldg(wv + m * G) * q, -g.w_clip), g.w_clip);
            const uint32_t qv = (__float_as_uint(q) & ~1u) | e;
            if (m < CMIN) sts32(base + m * kSlot, qv);
            else sts32_if(base + m * kSlot, qv, ln.has(P, m));
        }
        if (last) {   // slot 0 keeps L for the cut selection
            const uint32_t lv = (__float_as_uint(Lp) & ~1u) | e;
            if (CMIN > 0) sts32(base, lv);
            else sts32_if(base, lv, ln.has(P, 0));
        }
#ifdef BPDC_CHECKS
        if (!FAST && post_row && ((ln.vvalid >> P) & 1u) && !post_ok(g, (long long)P * G + u)) {} else
#endif
        if (!FAST && post_row && ((ln.vvalid >> P) & 1u)) post_row[__ldg(g.pos_col + P * G + u)] = Lp;
        return e;
    }

    // The variable updates of passes P .. PVM-1 (all passes of the variant on
    // the fast path, else those the graph occupies); ORs decision bit p of
    // each pass into nhd.
    template <bool FAST, int P>
    static __device__ __forceinline__ void var_passes(const DevGraph &g, const L &ln, int u, int t, bool last,
                                                      float *post_row, uint32_t &nhd)
    {
        if constexpr (P < PVM) {
            if (FAST || P < g.pv) nhd |= var_pass<FAST, P>(g, ln, u, t, last, post_row) << P;
            var_passes<FAST, P + 1>(g, ln, u, t, last, post_row, nhd);
        }
    }

    // One BP run (flooding, normalized min-sum).  The slots must hold the
    // initial messages, visible to the whole group.  Returns whether the hard
    // decision reproduced the syndrome; iters = iterations used; hd = hard
    // decision bits per variable pass.
    // FAST: every check and variable pass of the variant is occupied and no
    // posterior is written, so the per-pass guards compile away (the common
    // case of a graph packed for its own variant; identical arithmetic).
    template <bool FAST>
    static __device__ __forceinline__ bool run(const DevGraph &g, const L &ln, const Group<G> &grp,
                                               uint32_t sbits, uint32_t &hd, int &iters, float *post_row)
    {
        const int u = grp.u;
        const int T = g.max_iter;
        const float alpha = g.alpha;
        for (int t = 1;; ++t) {
            const bool scatter = t <= T;
            uint32_t unsat = 0;
            // ---- check phase ----
#pragma unroll
            for (int p = 0; p < PCM; ++p) {
                if constexpr (TAIL > 0) {
                    if (p == PCM - 1) {   // every lane takes part in the shared last pass
                        if (FAST || p < g.pc) unsat |= tail_pass(ln, p, sbits, alpha, scatter);
                        continue;
                    }
                }
                // on the fast path every check pass but the last is full, and
                // lanes without a check in the last pass skip it (their edges
                // all point at the +inf word, which keeps its value)
                if (FAST ? (p < PCM - 1 || ((ln.cvalid >> p) & 1u)) : p < g.pc) {
                    const bool live = (FAST && p < PCM - 1) || ((ln.cvalid >> p) & 1u);
                    // rows of up to 16 edges keep the gathered q in registers for
                    // the scatter; longer rows read each q again before
                    // overwriting it (one more load per edge, no register array)
                    constexpr bool kHold = DCM <= 16;
                    static_assert(kHold || RULE == 0, "product-sum rows are limited to 16 edges");
                    uint32_t qb[kHold ? DCM : 1];
                    // the syndrome bit enters as sign and parity: 0 or 0x80000001
                    // (a multiply, which the FMA pipe takes off the busy ALU pipe)
                    uint32_t S = ((sbits >> p) & 1u) * 0x80000001u;
                    if constexpr (RULE == 0) {
                        // normalized min-sum
                        float mn1 = f_inf(), mn2 = f_inf();
                        float qf[kHold ? DCM : 1];
                        float qh[L::kHoldLong ? DCM : 1];   // q of a long row (table form)
                        auto gather = [&](int k) {
                            // unused slots point at the group's +inf word
                            const float v = ldsf(ln.addr(p, k));
                            if constexpr (kHold) qf[k] = v;
                            S ^= __float_as_uint(v);   // bit 31: sign parity, bit 0: hard-decision parity
                            const float av = fabsf(v);
                            mn2 = fminf(mn2, fmaxf(mn1, av));
                            mn1 = fminf(mn1, av);
                        };
                        if constexpr (kHold) {
                            // edges in pairs: with lo <= hi the pair's
                            // smallest two, the second minimum of the four
                            // values {mn1 <= mn2, lo, hi} is
                            // min(mn2, max(mn1, lo), hi)
                            auto gather2 = [&](int k, bool first) {
                                const float va = ldsf(ln.addr(p, k)), vb = ldsf(ln.addr(p, k + 1));
                                qf[k] = va;
                                qf[k + 1] = vb;
                                S ^= __float_as_uint(va) ^ __float_as_uint(vb);
                                const float lo = fminf(fabsf(va), fabsf(vb)), hi = fmaxf(fabsf(va), fabsf(vb));
                                if (first) {
                                    mn1 = lo;
                                    mn2 = hi;
                                } else {
                                    mn2 = fmin3(mn2, fmaxf(mn1, lo), hi);
                                    mn1 = fminf(mn1, lo);
                                }
                            };
#pragma unroll
                            for (int k = 0; k + 1 < DCM; k += 2) gather2(k, k == 0);
                            if (DCM & 1) gather(DCM - 1);
                        } else if constexpr (L::kTab) {
                            // the lane's edge word indices come from its shared
                            // table, 8 per 16-byte load; the two edges of a word
                            // go through the pairwise minimum (mn1 = mn2 = +inf
                            // before the first pair gives the first pair's
                            // order statistics)
                            auto take = [&](float va, float vb) {
                                S ^= __float_as_uint(va) ^ __float_as_uint(vb);
                                const float lo = fminf(fabsf(va), fabsf(vb)), hi = fmaxf(fabsf(va), fabsf(vb));
                                mn2 = fmin3(mn2, fmaxf(mn1, lo), hi);
                                mn1 = fminf(mn1, lo);
                            };
                            auto take1 = [&](float v) {
                                S ^= __float_as_uint(v);
                                const float av = fabsf(v);
                                mn2 = fminf(mn2, fmaxf(mn1, av));
                                mn1 = fminf(mn1, av);
                            };
                            constexpr int kFull = DCM / kTabEdges, kTail = DCM % kTabEdges;
                            if constexpr (L::kHoldLong) {
                                // every chunk unrolled, the q of the row kept in qh
#pragma unroll
                                for (int c = 0; c < L::kTabChunks; ++c) {
                                    const uint4 w = lds128(ln.tab_entry(p, c));
                                    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                    for (int h = 0; h < 4; ++h) {
                                        const int k = c * kTabEdges + 2 * h;
                                        if (k + 1 < DCM) {
                                            qh[k] = ldsf(ln.word_addr(ww[h] & 0xFFFFu));
                                            qh[k + 1] = ldsf(ln.word_addr(ww[h] >> 16));
                                            take(qh[k], qh[k + 1]);
                                        } else if (k < DCM) {
                                            qh[k] = ldsf(ln.word_addr(ww[h] & 0xFFFFu));
                                            take1(qh[k]);
                                        }
                                    }
                                }
                            } else {
                                auto pair = [&](uint32_t w) {
                                    take(ldsf(ln.word_addr(w & 0xFFFFu)), ldsf(ln.word_addr(w >> 16)));
                                };
#pragma unroll 1
                                for (int c = 0; c < kFull; ++c) {
                                    const uint4 w = lds128(ln.tab_entry(p, c));
                                    pair(w.x);
                                    pair(w.y);
                                    pair(w.z);
                                    pair(w.w);
                                }
                                if constexpr (kTail > 0) {
                                    const uint4 w = lds128(ln.tab_entry(p, kFull));
                                    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                    for (int h = 0; h < kTail / 2; ++h) pair(ww[h]);
                                    if constexpr (kTail & 1) take1(ldsf(ln.word_addr(ww[kTail / 2] & 0xFFFFu)));
                                }
                            }
                        } else {   // long rows: bounded unrolling keeps few loads in flight
#pragma unroll 5
                            for (int k = 0; k < DCM; ++k) gather(k);
                        }
                        unsat |= S;
                        if (scatter) {
                            // the minimum over the other edges is min2 for the edge
                            // holding min1 and min1 for all others; with a tie at
                            // min1 both are equal, so no argmin is needed
                            // the row's sign parity rides on the scale factor
                            const float sa = __uint_as_float(__float_as_uint(alpha) ^ (S & 0x80000000u));
                            uint32_t m1 = __float_as_uint(scaled_min(sa, mn1));
                            uint32_t m2 = __float_as_uint(scaled_min(sa, mn2));
                            if (RC && !live) m1 = m2 = 0x7F800000u;   // idle check: writes +inf back
                            auto put = [&](int k) {
                                const uint32_t a = ln.addr(p, k);
                                float vk;
                                if constexpr (kHold) vk = qf[k];
                                else vk = ldsf(a);
                                const bool is_min = fabsf(vk) == mn1;
                                const uint32_t out = (is_min ? m2 : m1) ^ (__float_as_uint(vk) & 0x80000000u);
                                if (RC) sts32(a, out);
                                else sts32_if(a, out, a != ln.inf_addr);
                            };
                            if constexpr (kHold) {
#pragma unroll
                                for (int k = 0; k < DCM; ++k) put(k);
                            } else if constexpr (L::kTab) {
                                auto out_of = [&](float vk) {
                                    const bool is_min = fabsf(vk) == mn1;
                                    return (is_min ? m2 : m1) ^ (__float_as_uint(vk) & 0x80000000u);
                                };
                                auto store = [&](uint32_t a, uint32_t out) {
                                    if (RC) sts32(a, out);
                                    else sts32_if(a, out, a != ln.inf_addr);
                                };
                                constexpr int kFull = DCM / kTabEdges, kTail = DCM % kTabEdges;
                                if constexpr (L::kHoldLong) {
                                    // the held q decide each answer; the table gives the slots
#pragma unroll
                                    for (int c = 0; c < L::kTabChunks; ++c) {
                                        const uint4 w = lds128(ln.tab_entry(p, c));
                                        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                        for (int h = 0; h < 4; ++h) {
                                            const int k = c * kTabEdges + 2 * h;
                                            if (k < DCM) store(ln.word_addr(ww[h] & 0xFFFFu), out_of(qh[k]));
                                            if (k + 1 < DCM) store(ln.word_addr(ww[h] >> 16), out_of(qh[k + 1]));
                                        }
                                    }
                                } else {
                                    // each q read again from its slot, then overwritten by r
                                    auto put_at = [&](uint32_t a) { store(a, out_of(ldsf(a))); };
                                    auto put2 = [&](uint32_t w) {
                                        put_at(ln.word_addr(w & 0xFFFFu));
                                        put_at(ln.word_addr(w >> 16));
                                    };
#pragma unroll 1
                                    for (int c = 0; c < kFull; ++c) {
                                        const uint4 w = lds128(ln.tab_entry(p, c));
                                        put2(w.x);
                                        put2(w.y);
                                        put2(w.z);
                                        put2(w.w);
                                    }
                                    if constexpr (kTail > 0) {
                                        const uint4 w = lds128(ln.tab_entry(p, kFull));
                                        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                                        for (int h = 0; h < kTail / 2; ++h) put2(ww[h]);
                                        if constexpr (kTail & 1) put_at(ln.word_addr(ww[kTail / 2] & 0xFFFFu));
                                    }
                                }
                            } else {
#pragma unroll 5
                                for (int k = 0; k < DCM; ++k) put(k);
                            }
                        }
                    } else {
                        // product-sum: r_k = phi(sum_{j != k} phi(|q_j|)) with the
                        // extrinsic sign; +inf inputs (cut or unused) add phi = 0.
                        // The smallest argument of edge k's sum is min2 on the
                        // (unique) minimum edge and min1 on every other edge.
                        // With at most two finite inputs (min3 = +inf) every
                        // extrinsic set holds one finite value, and the rule
                        // returns it unchanged: that case takes the exact
                        // value instead of phi(phi(x)), which FP32 rounds.
                        float mn1 = f_inf(), mn2 = f_inf(), mn3 = f_inf();
#pragma unroll
                        for (int k = 0; k < DCM; ++k) {
                            const uint32_t b = lds32(ln.addr(p, k));
                            qb[k] = b;
                            S ^= b;
                            const float av = fabsf(__uint_as_float(b));
                            mn3 = fminf(mn3, fmaxf(mn2, av));
                            mn2 = fminf(mn2, fmaxf(mn1, av));
                            mn1 = fminf(mn1, av);
                        }
                        unsat |= S;
                        if (scatter) {
                            const bool pair = mn3 == f_inf();
                            const uint32_t Sm = S & 0x80000000u;
                            const float sa = fminf(fmaxf(mn1 - kPhiShift, 0.0f), kLlrCap);
                            const float sb = fminf(fmaxf(mn2 - kPhiShift, 0.0f), kLlrCap);
                            float f[DCM];
#pragma unroll
                            for (int k = 0; k < DCM; ++k) f[k] = phi(fabsf(__uint_as_float(qb[k])) - sa);
                            // the minimum edge's own sum, needed only when its
                            // shift differs (min2 > min1 and min2 > kPhiShift)
                            float rb = 0.0f;
                            if (sb != sa) {
                                float sum = 0.0f;
#pragma unroll
                                for (int k = 0; k < DCM; ++k) {
                                    const float av = fabsf(__uint_as_float(qb[k]));
                                    sum += av == mn1 ? 0.0f : phi(av - sb);
                                }
                                rb = sb + phi(sum);
                            }
                            float suf[DCM + 1];
                            suf[DCM] = 0.0f;
#pragma unroll
                            for (int k = DCM - 1; k >= 0; --k) suf[k] = suf[k + 1] + f[k];
                            float pre = 0.0f;
#pragma unroll
                            for (int k = 0; k < DCM; ++k) {
                                const uint32_t a = ln.addr(p, k);
                                const bool is_min = fabsf(__uint_as_float(qb[k])) == mn1;
                                const bool own_b = sb != sa && is_min;
                                float mag = pair ? scaled_min(1.0f, is_min ? mn2 : mn1)
                                                 : (own_b ? rb : sa + phi(pre + suf[k + 1]));
                                mag = fminf(mag, kLlrCap);
                                pre += f[k];
                                if (RC && !live) mag = f_inf();   // idle check: writes +inf back
                                uint32_t out = __float_as_uint(mag) ^ Sm ^ (qb[k] & 0x80000000u);
                                if (g.wts && live && a != ln.inf_addr) {   // weighted BP: r *= wc
#ifdef BPDC_CHECKS
                                    check_index(8, (long long)(min(t, g.w_T) - 1) * g.slots + ((a - ln.slot_base) >> 2), g.n_wts);
#endif
                                    const float w = __ldg(g.wts + (size_t)(min(t, g.w_T) - 1) * g.slots +
                                                          ((a - ln.slot_base) >> 2));
                                    out = __float_as_uint(w * __uint_as_float(out));
                                }
                                if (RC) sts32(a, out);
                                else sts32_if(a, out, a != ln.inf_addr);
                            }
                        }
                    }
                }
            }
            if (!grp.any((unsat & 1u) != 0)) { iters = t - 1; return true; }
            if (t > T) { iters = T; return false; }
            // ---- variable phase ----
            uint32_t nhd = 0;
            var_passes<FAST, 0>(g, ln, u, t, t == T, post_row, nhd);
            hd = nhd & ln.vvalid;
            grp.sync();
        }
    }

    static __device__ void decode(const LaunchDesc &ld, uint32_t *region, const Group<G> &grp, int gib)
    {
        const int u = grp.u;
        L ln;
        // little state lives across the iterations (the loop needs the
        // registers): shot indices are 32-bit (a launch holds fewer than 2^32
        // shots), and the current batch is an index into the launch's table
        int bi = -1;
        uint32_t bfirst = 0, bend = 0;
        // per-batch counters accumulate in the group's shared misc words 4..11
        // (lane 0 only) and are flushed when the group moves to another batch
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(region + 4);
        if (u == 0) cnt[0] = cnt[1] = cnt[2] = cnt[3] = 0;
        uint32_t bufsel = 0;
        const int groups_per_block = blockDim.x / G;
        bool once = false;
        bool lam_dirty = false;
        const uint32_t slot_base = (uint32_t)__cvta_generic_to_shared(region + kMiscWords);
        const uint32_t inf_word = (uint32_t)__cvta_generic_to_shared(region + 2);
        if (u == 0) region[2] = 0x7F800000u;   // read by unused check slots

        while (true) {
            // ---- next shot ----
            uint32_t w;
            if (ld.work) {
                unsigned long long x = 0;
                if constexpr (G <= 32) {
                    if (u == 0) x = atomicAdd((unsigned long long *)ld.work, 1ull);
                    x = __shfl_sync(grp.mask, x, grp.leader);
                } else {
                    // the ticket goes through a shared word (two, alternating);
                    // drawn only when the group is free, so that a shot never
                    // waits behind a long one on a busy group.  This barrier
                    // also keeps a fast lane from writing the next shot's slots
                    // or staging (of another graph, perhaps) before every lane
                    // has copied out the previous shot
                    uint32_t *misc = region + 0;
                    if (u == 0) misc[bufsel] = (uint32_t)atomicAdd((unsigned long long *)ld.work, 1ull);
                    grp.sync();
                    x = misc[bufsel];
                    bufsel ^= 1u;
                }
                w = (uint32_t)x;
            } else {
                if (once) break;
                once = true;
                w = blockIdx.x * (uint32_t)groups_per_block + (uint32_t)gib;
            }
            if ((int64_t)w >= ld.total) break;
            if (w < bfirst || w >= bend) {
                if (u == 0) {
                    if (bi >= 0 && ld.batches[bi].counters)
                        for (int x = 0; x < 4; ++x) atomicAdd(ld.batches[bi].counters + x, cnt[x]);
                    cnt[0] = cnt[1] = cnt[2] = cnt[3] = 0;
                }
                int lo = 0, hi = ld.n_batches - 1;
                while (lo < hi) {  // last batch with first <= w
                    const int mid = (lo + hi + 1) >> 1;
                    if (ld.batches[mid].first <= (int64_t)w) lo = mid; else hi = mid - 1;
                }
                const DevGraph &gnew = ld.batches[lo].g;
                if (bi < 0 || gnew.chk_idx != ld.batches[bi].g.chk_idx || gnew.lam != ld.batches[bi].g.lam) {
                    ln.load(gnew, u, slot_base, inf_word);
                    lam_dirty = false;
                }
                bi = lo;
                bfirst = (uint32_t)ld.batches[bi].first;
                bend = bfirst + (uint32_t)ld.batches[bi].B;
            }
            const BatchDesc &bd = ld.batches[bi];
            // the graph's fields are read where they are used (L1 hits), not
            // copied per shot: a copy of the whole descriptor took registers
            // and stack from the iterations (2-10 % slower)
            const DevGraph &g = bd.g;
            const uint32_t b = w - bfirst;
            uint32_t *cm = region + kMiscWords + g.slots;   // cut mask, then e_hat staging
            uint32_t *ls = cm + g.cmw;               // logical-flip staging
            float *post_row = bd.post ? bd.post + (size_t)b * g.N : nullptr;
            const uint32_t *cut_in = bd.cut_in;
            if (lam_dirty) { ln.reload_lam(g, u); lam_dirty = false; }

            // ---- a1: syndrome bits of my checks ----
            uint32_t sbits = 0;
            const uint32_t *sy = bd.syn + (size_t)b * g.MW;
#pragma unroll
            for (int p = 0; p < PCM; ++p) {
                // a shared last pass: the first lane of each check holds its bit
                const bool tail = TAIL > 0 && p == PCM - 1;
                const int i = tail ? p * G + u / (TAIL > 0 ? TAIL : 1) : p * G + u;
                const bool own = !tail || u % (TAIL > 0 ? TAIL : 1) == 0;
                if (p < g.pc && i < g.M && own) sbits |= ((__ldg(sy + (i >> 5)) >> (i & 31)) & 1u) << p;
            }
            uint32_t hd = 0;
            int st = 0, it1 = 0, it2 = 0;
            bool ran_dc = false;
            if (cut_in) {
                // BP on a given cut graph (Algorithm 2 form), no DC: cut priors -> +inf
                const uint32_t *ci = cut_in + (size_t)b * g.NW;
#pragma unroll
                for (int p = 0; p < PVM; ++p) {
                    const int j = p * G + u;
                    const int c = (p < g.pv && ((ln.vvalid >> p) & 1u)) ? __ldg(g.pos_col + j) : -1;
                    if (c >= 0 && ((__ldg(ci + (c >> 5)) >> (c & 31)) & 1u)) {
                        ln.lamv[p] = f_inf();
                        lam_dirty = true;
                    }
                }
            }
            // initial messages of the first run (also writes the prior as the
            // posterior when one is requested), and the correction and
            // logical-flip staging cleared (each lane the words it copies out
            // in the epilogue); the vote is the barrier that publishes both
            hd = init(g, ln, u, post_row);
            for (int x = u; x < g.NW; x += G) cm[x] = 0;
            for (int x = u; x < g.KW; x += G) ls[x] = 0;
            const bool nonzero = grp.any(sbits != 0);
            if (!cut_in && !nonzero && g.zero_ok) {
                // converged before the first iteration: e_hat = 0 (every prior < 1/2)
                hd = 0;
            } else {
                for (bool second = false;; second = true) {
                    if (second) {
                        hd = init(g, ln, u, post_row);
                        grp.sync();
                    }
                    int iters = 0;
                    const bool ok = (g.pc == PCM && g.pv == PVM && !post_row)
                                        ? run<true>(g, ln, grp, sbits, hd, iters, post_row)
                                        : run<false>(g, ln, grp, sbits, hd, iters, post_row);
                    if (second) it2 = iters; else it1 = iters;
                    if (ok) { st = second ? 1 : 0; break; }
                    if (second || cut_in || !g.dc_enable) { st = 2; break; }
                    // ---- a7: cut selection on the last posterior (slot 0) ----
                    ran_dc = true;
                    for (int x = u; x < g.cmw; x += G) cm[x] = 0;
                    grp.sync();
                    cut_rows(
                        g, bd.shot_offset + (uint64_t)b, u, G,
                        [&](int, uint32_t e) {
                            const uint32_t s0 = e & 0xFFFFu;
#ifdef BPDC_CHECKS
                            if (s0 == kNoEdge ? !check_index(5, e >> 16, g.n_pos) : !check_index(1, s0, g.slots)) return f_inf();
#endif
                            return s0 == kNoEdge ? __ldg(g.lam + (e >> 16)) : ldsf(slot_base + 4u * s0);
                        },
                        [&](int, uint32_t e) { atomicOr(cm + ((e >> 16) >> 5), 1u << ((e >> 16) & 31)); });
                    grp.sync();
#pragma unroll
                    for (int p = 0; p < PVM; ++p) {
                        const int j = p * G + u;
                        if (p < g.pv && ((ln.vvalid >> p) & 1u)) {
                            if ((cm[j >> 5] >> (j & 31)) & 1u) {
                                ln.lamv[p] = f_inf();   // Algorithm 2: cut prior 0
                            } else if (g.dc_prior && ln.has(p, 0)) {
                                // first-run posterior as prior, p_hat clamped to [1e-12, 1/2]
                                const float Lj = __uint_as_float(
                                    __float_as_uint(ldsf(slot_base + 4u * (uint32_t)(L::off(p) * G + u))) & ~1u);
                                ln.lamv[p] = fminf(fmaxf(Lj, 0.0f), 27.631021115928547f);
                            }
                        }
                    }
                    lam_dirty = true;
                    grp.sync();
                    // the staging again (it held the cut mask), published by the
                    // barrier after the second run's initial messages
                    for (int x = u; x < g.cmw; x += G) cm[x] = 0;
                    // ---- a8: BP again on the cut graph ----
                }
            }

            // ---- a9: epilogue ----
            // corrections and logical flips from the set decision bits into the
            // cleared staging (shared atomics), published by one barrier
            uint32_t *corr = bd.corr + (size_t)b * g.NW;
#pragma unroll
            for (int p = 0; p < PVM; ++p) {
                if ((hd >> p) & 1u) {
                    const int j = p * G + u;
                    const int c = __ldg(g.pos_col + j);
#ifdef BPDC_CHECKS
                    if (!check_index(7, c, g.N)) continue;
#endif
                    atomicOr(cm + (c >> 5), 1u << (c & 31));
                    const uint32_t *lc = g.l_bits + (size_t)j * g.KW;
                    for (int x = 0; x < g.KW; ++x) {
                        const uint32_t v = __ldg(lc + x);
                        if (v) atomicXor(ls + x, v);
                    }
                }
            }
            grp.sync();
            bool fail_local = false;
            for (int x = u; x < g.NW; x += G) corr[x] = cm[x];
            for (int x = u; x < g.KW; x += G) {
                const uint32_t v = ls[x];
                if (bd.lflips) bd.lflips[(size_t)b * g.KW + x] = v;
                if (bd.obs_true && __ldg(bd.obs_true + (size_t)b * g.KW + x) != v) fail_local = true;
            }
            // a logical flip differing from the true one: the lanes holding
            // logical words are the group's first warp when there are at most
            // 32 of them, so a warp vote suffices there
            bool fail_obs;
            if constexpr (G > 32) {
                if (g.KW <= 32) {
                    const bool v = u < 32 ? __any_sync(0xFFFFFFFFu, fail_local) != 0 : false;
                    fail_obs = v;
                } else {
                    fail_obs = grp.any(fail_local);
                }
            } else {
                fail_obs = grp.any(fail_local);
            }
            const bool fail = fail_obs || st == 2;
            if (u == 0) {
                bd.status[b] = (uint8_t)st;
                if (bd.iters) bd.iters[b] = (uint32_t)it1 | ((uint32_t)it2 << 16);
                cnt[0] += 1;
                cnt[1] += fail ? 1 : 0;
                cnt[2] += (unsigned long long)(it1 + it2);
                cnt[3] += ran_dc ? 1 : 0;
            }
        }
        if (bi >= 0 && u == 0 && ld.batches[bi].counters)
            for (int x = 0; x < 4; ++x) atomicAdd(ld.batches[bi].counters + x, cnt[x]);
    }
};

template <int G, int PCM, int DCM, int PVM, int CVM, int CMIN, bool RC, int RULE, int BLOCK, int MINB,
          uint64_t PROF, bool TAB, int TAIL>
__global__ void __launch_bounds__(BLOCK, MINB) decode_kernel(LaunchDesc ld, int region_words)
{
    extern __shared__ uint32_t smem[];
    const int tid = threadIdx.x;
    const int gib = tid / G;
    Group<G> grp;
    grp.u = tid % G;
    grp.bar = 1 + gib;
    if constexpr (G <= 32) {
        const int wl = tid & 31;
        const int base = (wl / G) * G;
        grp.mask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << base);
        grp.leader = base;
    } else {
        grp.mask = 0xFFFFFFFFu;
        grp.leader = 0;
    }
    uint32_t *region = smem + (size_t)gib * region_words;
    Decoder<G, PCM, DCM, PVM, CVM, CMIN, RC, RULE, PROF, TAB, TAIL>::decode(ld, region, grp, gib);
}

// Cut selection alone, one block per shot (same selection code as the fused kernel).
__global__ void cut_select_kernel(DevGraph g, int64_t B, const float *post, uint64_t shot_offset,
                                  uint32_t *cut_out)
{
    extern __shared__ uint32_t sm[];
    uint32_t *cm = sm;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        for (int x = threadIdx.x; x < g.NW; x += blockDim.x) cm[x] = 0;
        __syncthreads();
        const float *row = post + (size_t)b * g.N;
        cut_rows(
            g, shot_offset + (uint64_t)b, threadIdx.x, blockDim.x,
            [&](int a, uint32_t) { return __ldg(row + __ldg(g.d_col + a)); },
            [&](int a, uint32_t) {
                const int c = __ldg(g.d_col + a);
                atomicOr(cm + (c >> 5), 1u << (c & 31));
            });
        __syncthreads();
        for (int x = threadIdx.x; x < g.NW; x += blockDim.x) cut_out[(size_t)b * g.NW + x] = cm[x];
        __syncthreads();
    }
}

// Seeded sampler: errors, syndromes e H^T and observables e L^T, one block per shot.
__global__ void sample_kernel(DevGraph g, int64_t B, uint64_t seed, uint64_t shot_offset,
                              uint32_t *syn, uint32_t *obs, uint32_t *err)
{
    extern __shared__ uint32_t sm[];
    uint32_t *eb = sm, *sb = sm + g.NW, *ob = sb + g.MW;
    const int nw = g.NW + g.MW + g.KW;
    for (int64_t b = blockIdx.x; b < B; b += gridDim.x) {
        for (int x = threadIdx.x; x < nw; x += blockDim.x) sm[x] = 0;
        __syncthreads();
        const uint64_t gs = shot_offset + (uint64_t)b;
        for (int j = threadIdx.x; j < g.N; j += blockDim.x) {
            const uint64_t h = splitmix64(seed, gs * (uint64_t)g.N + (uint64_t)j);
            if ((uint32_t)(h >> 32) < __ldg(g.thr + j)) atomicOr(eb + (j >> 5), 1u << (j & 31));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < g.M; i += blockDim.x) {
            uint32_t par = 0;
            for (int a = __ldg(g.h_ptr + i); a < __ldg(g.h_ptr + i + 1); ++a) {
                const int c = __ldg(g.h_col + a);
                par ^= (eb[c >> 5] >> (c & 31)) & 1u;
            }
            if (par) atomicOr(sb + (i >> 5), 1u << (i & 31));
        }
        for (int j = threadIdx.x; j < g.N; j += blockDim.x) {
            if ((eb[j >> 5] >> (j & 31)) & 1u) {
                for (int x = 0; x < g.KW; ++x) {
                    const uint32_t v = __ldg(g.l_col + (size_t)j * g.KW + x);
                    if (v) atomicXor(ob + x, v);
                }
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < g.MW; x += blockDim.x) syn[(size_t)b * g.MW + x] = sb[x];
        if (obs)
            for (int x = threadIdx.x; x < g.KW; x += blockDim.x) obs[(size_t)b * g.KW + x] = ob[x];
        if (err)
            for (int x = threadIdx.x; x < g.NW; x += blockDim.x) err[(size_t)b * g.NW + x] = eb[x];
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Variant table: (id, G, check passes, row weight, variable passes, column
// weight, minimum column weight, regular rows, check rule (0 min-sum,
// 1 product-sum), block threads, min blocks per SM, slots per variable pass
// (3 bits per pass, 0: the column weight in every pass), shared edge table,
// lanes per check of a shared last check pass (0: none)).
// Variants 13 and 14 take circuit-level detector models (rows of up to 35
// edges, one shot per SM): 13 with 6 slots in every pass and the check-edge
// indices read from global memory at each access, 14 with variables sorted by
// degree into passes of 6, 5, 4, 3, ... slots (a third less shared memory)
// and the check-edge indices in a shared-memory table.  Variant 15 is variant
// 1 (HGP-like graphs) with passes of 4, 4, 4, 4, 3, ... slots: the degree-4
// variables of a hypergraph product in the first passes.  Variant 16 is the
// circuit-level form with 512 threads per shot (two check passes, 18
// variable passes of 6, 6, 5, 5, 4, 4, 3, ..., 3, 2 slots): at 128 registers
// a thread keeps its row's 35 gathered q for the scatter instead of reading
// them again.  Variants 17 and 18 have the shape of BB[[72,12,6]] (two check
// and three variable passes of a warp: its fast path) at 4 and 6 blocks per SM.
// Variants 19 and 20 are variants 17 and 7 with the last check pass shared
// (BB[[72,12,6]]: its 4 checks past the first 32 on 8 lanes each;
// BB[[144,12,12]]: its 8 checks past the first 64 on 4 lanes each).
#define BPDC_VARIANTS(X)                                                       \
    X(0, 32, 3, 6, 5, 3, 3, true, 0, 256, 4, 0, false, 0)                      \
    X(1, 256, 5, 7, 10, 4, 3, true, 0, 256, 3, 0, false, 0)                    \
    X(2, 512, 3, 7, 5, 4, 3, true, 0, 512, 2, 0, false, 0)                     \
    X(3, 256, 4, 8, 11, 3, 2, false, 0, 256, 3, 0, false, 0)                   \
    X(4, 512, 2, 8, 6, 3, 2, false, 0, 512, 2, 0, false, 0)                    \
    X(5, 32, 4, 8, 8, 4, 1, false, 0, 256, 4, 0, false, 0)                     \
    X(6, 128, 10, 7, 20, 4, 3, true, 0, 128, 6, 0, false, 0)                   \
    X(7, 32, 3, 6, 5, 3, 3, true, 0, 256, 3, 0, false, 0)                      \
    X(8, 256, 5, 7, 10, 4, 3, true, 0, 256, 2, 0, false, 0)                    \
    X(9, 512, 3, 7, 5, 4, 3, true, 0, 512, 1, 0, false, 0)                     \
    X(10, 256, 4, 8, 11, 3, 2, false, 0, 256, 2, 0, false, 0)                  \
    X(11, 32, 4, 4, 4, 2, 1, false, 1, 256, 4, 0, false, 0)                    \
    X(12, 32, 3, 6, 5, 3, 3, true, 1, 256, 4, 0, false, 0)                     \
    X(13, 1024, 1, 35, 9, 6, 2, false, 0, 1024, 1, 0, false, 0)                \
    X(14, 1024, 1, 35, 9, 6, 2, false, 0, 1024, 1, 0x36db72eull, true, 0)      \
    X(15, 256, 5, 7, 10, 4, 3, true, 0, 256, 3, 0x1b6db924ull, false, 0)       \
    X(16, 512, 2, 35, 18, 6, 2, false, 0, 512, 1, 0x136db6db6e4b76ull, true, 0) \
    X(17, 32, 2, 6, 3, 3, 3, true, 0, 256, 4, 0, false, 0)                     \
    X(18, 32, 2, 6, 3, 3, 3, true, 0, 256, 6, 0, false, 0)                     \
    X(19, 32, 2, 6, 3, 3, 3, true, 0, 256, 4, 0, false, 8)                     \
    X(20, 32, 3, 6, 5, 3, 3, true, 0, 256, 3, 0, false, 4)

static const Variant kVariants[] = {
#define X(id, G, PC, DC, PV, CV, CMIN, RC, RULE, BLK, MB, PROF, TAB, TAIL) \
    {id, G, PC, DC, PV, CV, CMIN, RC, RULE, BLK, MB, PROF, TAB, TAIL},
    BPDC_VARIANTS(X)
#undef X
};

int num_variants() { return (int)(sizeof(kVariants) / sizeof(kVariants[0])); }
const Variant &variant(int id) { return kVariants[id]; }

#ifdef BPDC_CHECKS
bool check_status(int *site, long long *index)
{
    unsigned long long v[2] = {0ull, 0ull};
    if (cudaMemcpyFromSymbol(v, g_check, sizeof(v)) != cudaSuccess) return false;
    const unsigned long long z[2] = {0ull, 0ull};
    if (cudaMemcpyToSymbol(g_check, z, sizeof(z)) != cudaSuccess) return false;
    *site = (int)v[0];
    *index = (long long)v[1];
    return true;
}
#else
bool check_status(int *, long long *) { return false; }
#endif

static const void *variant_fn(int id)
{
    switch (id) {
#define X(id, G, PC, DC, PV, CV, CMIN, RC, RULE, BLK, MB, PROF, TAB, TAIL) \
    case id: return (const void *)decode_kernel<G, PC, DC, PV, CV, CMIN, RC, RULE, BLK, MB, PROF, TAB, TAIL>;
        BPDC_VARIANTS(X)
#undef X
    default: return nullptr;
    }
}

// Occupancy of a variant at a shared-memory size, cached per device.  The
// dynamic shared-memory limit of a kernel only ever grows, so a smaller graph
// created later never lowers it under a larger one that is still in use.
cudaError_t variant_attributes(int id, int smem_bytes, int *blocks_per_sm, int *regs)
{
    const void *fn = variant_fn(id);
    if (!fn) return cudaErrorInvalidValue;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::mutex mu;
    static std::map<std::tuple<int, int, int>, std::pair<int, int>> cache;   // (dev, id, smem) -> (bps, regs)
    static std::map<std::pair<int, int>, int> limit;                         // (dev, id) -> smem limit set
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(std::make_tuple(dev, id, smem_bytes));
    if (it != cache.end()) {
        *blocks_per_sm = it->second.first;
        if (regs) *regs = it->second.second;
        return cudaSuccess;
    }
    int &lim = limit[std::make_pair(dev, id)];
    if (smem_bytes > lim) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
        if (e != cudaSuccess) return e;
        lim = smem_bytes;
    }
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kVariants[id].block_threads, smem_bytes);
    if (e != cudaSuccess) return e;
    cache[std::make_tuple(dev, id, smem_bytes)] = std::make_pair(bps, (int)fa.numRegs);
    *blocks_per_sm = bps;
    if (regs) *regs = fa.numRegs;
    return cudaSuccess;
}

cudaError_t launch_variant(int id, const LaunchDesc &ld, int grid, int smem_bytes, cudaStream_t s)
{
    const int region = smem_bytes / 4 / (kVariants[id].block_threads / kVariants[id].G);
    switch (id) {
#define X(id, G, PC, DC, PV, CV, CMIN, RC, RULE, BLK, MB, PROF, TAB, TAIL)                          \
    case id:                                                                                        \
        decode_kernel<G, PC, DC, PV, CV, CMIN, RC, RULE, BLK, MB, PROF, TAB, TAIL>                  \
            <<<grid, BLK, smem_bytes, s>>>(ld, region);                                             \
        return cudaGetLastError();
        BPDC_VARIANTS(X)
#undef X
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Allocation-free launches.  The persistent decode kernel needs a little
// global scratch besides its inputs and outputs: the device work counter and
// the descriptors of the batches of one launch.  bpdc_decode_multi takes it
// from the graph's preallocated ring; the allocation-free entry point takes it
// from this fixed array instead, which every GPU that loads the library keeps
// until the process exits.  Every call shares it and it keeps the contents of
// the last call; calls whose launches overlap on the GPU race on it.
static __device__ __align__(256) unsigned char g_static_scratch[256 + kStaticBatches * sizeof(BatchDesc)];

// Device address of the scratch array on the current device.  In host code
// the symbol is only a host-side stand-in; the address comes from
// cudaGetSymbolAddress, resolved once per device with that device current.
// Calls from several host threads may resolve it at the same time: they store
// the same value, through atomics.
static cudaError_t static_scratch_address(void **out)
{
    constexpr int kMaxDevices = 64;
    static std::atomic<void *> addr[kMaxDevices];
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void *p = addr[dev].load(std::memory_order_acquire);
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

// Descriptors of an allocation-free launch, passed by value: the launch
// copies them into its parameter buffer, so a captured CUDA graph replays
// them without reading host memory again.
struct StaticSetup {
    BatchDesc d[kStaticBatches];
    int n;
};

__global__ void static_setup_kernel(StaticSetup st, BatchDesc *dst, unsigned long long *work)
{
    const int i = threadIdx.x;
    if (i < st.n) dst[i] = st.d[i];
    if (i == 0) *work = 0ull;   // the work counter starts at zero
}

cudaError_t launch_variant_static(int id, const BatchDesc *host_descs, int n, int64_t total, int grid,
                                  int smem_bytes, cudaStream_t s)
{
    if (n < 1 || n > kStaticBatches) return cudaErrorInvalidValue;
    void *base = nullptr;
    cudaError_t e = static_scratch_address(&base);
    if (e != cudaSuccess) return e;
    auto *work = reinterpret_cast<unsigned long long *>(base);
    auto *descs = reinterpret_cast<BatchDesc *>(static_cast<unsigned char *>(base) + 256);
    StaticSetup st;
    for (int i = 0; i < n; ++i) st.d[i] = host_descs[i];
    st.n = n;
    static_setup_kernel<<<1, 32, 0, s>>>(st, descs, work);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    LaunchDesc ld{};
    ld.batches = descs;
    ld.n_batches = n;
    ld.total = total;
    ld.work = reinterpret_cast<unsigned int *>(work);
    return launch_variant(id, ld, grid, smem_bytes, s);
}

cudaError_t launch_cut_select(const DevGraph &g, int64_t B, const float *post, uint64_t shot_offset,
                              uint32_t *cut_out, cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    const int grid = (int)(B < 65536 ? B : 65536);
    cut_select_kernel<<<grid, 256, g.NW * 4, s>>>(g, B, post, shot_offset, cut_out);
    return cudaGetLastError();
}

cudaError_t launch_sample(const DevGraph &g, int64_t B, uint64_t seed, uint64_t shot_offset,
                          uint32_t *syn, uint32_t *obs, uint32_t *err, cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    const int smem = (g.NW + g.MW + g.KW) * 4;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void *)sample_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (int)(B < 152 * 16 ? B : 152 * 16);
    sample_kernel<<<grid, 256, smem, s>>>(g, B, seed, shot_offset, syn, obs, err);
    return cudaGetLastError();
}

}  // namespace bpdc
