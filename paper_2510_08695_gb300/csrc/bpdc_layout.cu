// Host-side placement of Tanner-graph variables and ordering of check edges
// for conflict-free shared-memory access.
//
// In the message layout every slot of the variable at position pos lies in
// bank pos mod 32 (positions are p*G + u with G a multiple of 32).  The check
// update of one warp handles 32 consecutive checks (a "group") and, in round k,
// gathers and scatters the k-th edge of each: the round is conflict-free when
// those 32 edges lie in 32 distinct banks.  Two choices are free and change no
// arithmetic:
//   1. which bank class each variable gets (its position mod 32): a local
//      search (single moves under the per-bank capacity, then swaps) lowers,
//      for every group, the number of edges a bank receives beyond the
//      group's row weight;
//   2. the order of the edges inside each check: per group, a proper edge
//      colouring of the bipartite multigraph checks x banks with dc colours
//      (Konig's theorem: bipartite multigraphs of maximum degree dc are
//      dc-edge-colourable; built with alternating-path recolouring); a bank
//      with more than dc edges in a group is split into virtual nodes of at
//      most dc edges, whose copies then share rounds (unavoidable conflicts).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "bpdc_internal.h"

namespace bpdc {
namespace {

// Deterministic xorshift for the local search order.
struct Rng {
    uint64_t s;
    explicit Rng(uint64_t seed) : s(seed * 0x9E3779B97F4A7C15ull + 1) {}
    uint32_t next()
    {
        s ^= s << 13;
        s ^= s >> 7;
        s ^= s << 17;
        return (uint32_t)(s >> 16);
    }
};

// cap: variables per bank.  cap_ge (empty: none): cap_ge[d] is the most
// variables of degree >= d one bank may hold (its positions in passes with at
// least d slots).
void assign_banks(int M, int N, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col,
                  int cap, const std::vector<int> &cap_ge, std::vector<int> &bank)
{
    const int ng = (M + 31) / 32;
    std::vector<int> d(ng, 0);
    for (int i = 0; i < M; ++i) d[i / 32] = std::max(d[i / 32], row_ptr[i + 1] - row_ptr[i]);
    // groups touched by each variable, once each, with the number of edges
    std::vector<std::vector<std::pair<int, int>>> vg(N);
    for (int i = 0; i < M; ++i)
        for (int a = row_ptr[i]; a < row_ptr[i + 1]; ++a) {
            auto &l = vg[col[a]];
            if (!l.empty() && l.back().first == i / 32) l.back().second++;
            else l.emplace_back(i / 32, 1);
        }
    // variables of each group (with multiplicity), for the annealing
    std::vector<std::vector<int>> gv(ng);
    for (int i = 0; i < M; ++i)
        for (int a = row_ptr[i]; a < row_ptr[i + 1]; ++a) gv[i / 32].push_back(col[a]);
    // degree of every variable, and per bank the number of members of degree >= d
    std::vector<int> deg(N, 0);
    for (int32_t c : col) deg[c]++;
    const int dmax = cap_ge.empty() ? 0 : (int)cap_ge.size() - 1;
    std::vector<int> ge((size_t)32 * (dmax + 1), 0);
    bank.resize(N);
    if (cap_ge.empty()) {
        for (int j = 0; j < N; ++j) bank[j] = j % 32;
    } else {
        // start balanced: variables in order of decreasing degree, dealt round robin
        std::vector<int> byd(N);
        std::iota(byd.begin(), byd.end(), 0);
        std::stable_sort(byd.begin(), byd.end(), [&](int a, int b) { return deg[a] > deg[b]; });
        for (int r = 0; r < N; ++r) bank[byd[r]] = r % 32;
        for (int j = 0; j < N; ++j)
            for (int d = 1; d <= std::min(deg[j], dmax); ++d) ge[(size_t)bank[j] * (dmax + 1) + d]++;
    }
    // j may join bank b (which does not hold it) without a swap
    auto fits = [&](int j, int b) {
        for (int d = 1; d <= std::min(deg[j], dmax); ++d)
            if (ge[(size_t)b * (dmax + 1) + d] + 1 > cap_ge[d]) return false;
        return true;
    };
    // j (in b0) and j2 (in b) may trade banks
    auto fits_swap = [&](int j, int b0, int j2, int b) {
        const int lo = std::min(deg[j], deg[j2]), hi = std::min(std::max(deg[j], deg[j2]), dmax);
        const int gain = deg[j] > deg[j2] ? b : b0;   // the bank that takes the higher degree
        for (int d = lo + 1; d <= hi; ++d)
            if (ge[(size_t)gain * (dmax + 1) + d] + 1 > cap_ge[d]) return false;
        return true;
    };
    std::vector<int> n((size_t)ng * 32, 0);
    for (int j = 0; j < N; ++j)
        for (auto gc : vg[j]) n[(size_t)gc.first * 32 + bank[j]] += gc.second;
    std::vector<std::vector<int>> members(32);
    std::vector<int> slot_in(N);
    for (int j = 0; j < N; ++j) {
        slot_in[j] = (int)members[bank[j]].size();
        members[bank[j]].push_back(j);
    }
    auto over = [&](int g, int x) { return std::max(0, x - d[g]); };
    // cost change of moving j from b0 to b (n unchanged)
    auto delta = [&](int j, int b0, int b) {
        int dl = 0;
        for (auto gc : vg[j]) {
            const int g = gc.first, c = gc.second;
            const int x0 = n[(size_t)g * 32 + b0], x1 = n[(size_t)g * 32 + b];
            dl += over(g, x0 - c) - over(g, x0) + over(g, x1 + c) - over(g, x1);
        }
        return dl;
    };
    auto move = [&](int j, int b0, int b) {
        for (auto gc : vg[j]) {
            n[(size_t)gc.first * 32 + b0] -= gc.second;
            n[(size_t)gc.first * 32 + b] += gc.second;
        }
        for (int d = 1; d <= std::min(deg[j], dmax); ++d) {
            ge[(size_t)b0 * (dmax + 1) + d]--;
            ge[(size_t)b * (dmax + 1) + d]++;
        }
        auto &m0 = members[b0];
        const int last = m0.back();
        m0[slot_in[j]] = last;
        slot_in[last] = slot_in[j];
        m0.pop_back();
        slot_in[j] = (int)members[b].size();
        members[b].push_back(j);
        bank[j] = b;
    };
    // best move of j out of b0 (into a bank with room) or swap with a sampled
    // member of a full bank; returns the cost change, bt / jt the choice
    Rng rng(2510);
    auto best_move = [&](int j, int b0, int swaps, int &bt, int &jt) {
        int best = 1 << 30;
        bt = jt = -1;
        for (int b = 0; b < 32; ++b) {
            if (b == b0) continue;
            if ((int)members[b].size() < cap && (cap_ge.empty() || fits(j, b))) {
                const int dl = delta(j, b0, b);
                if (dl < best || (dl == best && (rng.next() & 1))) { best = dl; bt = b; jt = -1; }
            } else {
                const auto &mb = members[b];
                for (int s = 0; s < swaps && !mb.empty(); ++s) {
                    const int j2 = mb[rng.next() % mb.size()];
                    if (!cap_ge.empty() && !fits_swap(j, b0, j2, b)) continue;
                    const int d1 = delta(j, b0, b);
                    move(j, b0, b);
                    const int d2 = delta(j2, b, b0);
                    move(j, b, b0);
                    if (d1 + d2 < best || (d1 + d2 == best && (rng.next() & 1))) { best = d1 + d2; bt = b; jt = j2; }
                }
            }
        }
        return best;
    };
    // 1. descent: every variable in turn takes its best strictly improving move
    std::vector<int> order(N);
    std::iota(order.begin(), order.end(), 0);
    for (int round = 0; round < 60; ++round) {
        for (int k = N - 1; k > 0; --k) std::swap(order[k], order[rng.next() % (k + 1)]);
        int improved = 0;
        for (int j : order) {
            const int b0 = bank[j];
            int bt, jt;
            if (best_move(j, b0, 6, bt, jt) < 0) {
                move(j, b0, bt);
                if (jt >= 0) move(jt, bt, b0);
                ++improved;
            }
        }
        if (!improved) break;
    }
    // 2. simulated annealing aimed at the overloaded (group, bank) cells: a
    // variable of such a cell takes its best move even when that raises the
    // overflow, with probability exp(-increase / T) under a falling
    // temperature; the best assignment seen is kept.  The budget grows with
    // the number of variables (deterministic: fixed seed and iteration count).
    long cost = 0;
    for (int g = 0; g < ng; ++g)
        for (int b = 0; b < 32; ++b) cost += over(g, n[(size_t)g * 32 + b]);
    long best_cost = cost;
    std::vector<int> best_bank = bank;
    const long iters = std::min<long>(3000000L, 400L * N);
    const double T0 = 0.7;
    std::vector<int> hot;
    for (long it = 0; it < iters && cost > 0; ++it) {
        if ((it & 255) == 0 || hot.empty()) {
            hot.clear();
            for (int c = 0; c < ng * 32; ++c)
                if (n[c] > d[c / 32]) hot.push_back(c);
            if (hot.empty()) break;
        }
        const int cell = hot[rng.next() % hot.size()];
        const int g = cell / 32, b0 = cell % 32;
        if (n[cell] <= d[g]) continue;
        int j = -1;
        for (int tries = 0; tries < 64 && j < 0; ++tries) {
            const int jj = gv[g][rng.next() % gv[g].size()];
            if (bank[jj] == b0) j = jj;
        }
        if (j < 0) continue;
        int bt, jt;
        const int dl = best_move(j, b0, 16, bt, jt);
        if (bt < 0) continue;
        const double T = T0 * (1.0 - (double)it / (double)iters) + 1e-3;
        if (dl <= 0 || (double)(rng.next() & 0xFFFF) * (1.0 / 65536.0) < std::exp(-dl / T)) {
            move(j, b0, bt);
            if (jt >= 0) move(jt, bt, b0);
            cost += dl;
            if (cost < best_cost) {
                best_cost = cost;
                best_bank = bank;
            }
        }
    }
    bank = best_bank;
}

// Konig colouring of one group's bipartite multigraph; left = checks (local
// index), right = virtual banks.  edges: (left, right); returns colour per edge.
std::vector<int> color_group(int nl, int nr, int D, const std::vector<std::pair<int, int>> &edges)
{
    const int E = (int)edges.size();
    std::vector<int> atL((size_t)nl * D, -1), atR((size_t)nr * D, -1), colr(E, -1);
    for (int e = 0; e < E; ++e) {
        const int l = edges[e].first, r = edges[e].second;
        int a = -1, b = -1;
        for (int c = 0; c < D && a < 0; ++c)
            if (atL[(size_t)l * D + c] < 0) a = c;
        for (int c = 0; c < D && b < 0; ++c)
            if (atR[(size_t)r * D + c] < 0) b = c;
        if (a < 0 || b < 0) continue;   // cannot happen when degrees are <= D
        if (atR[(size_t)r * D + a] >= 0) {
            // flip the a/b alternating path that starts at r with colour a
            std::vector<int> path;
            int node = r;
            bool right = true;
            int c = a;
            while (true) {
                const int f = right ? atR[(size_t)node * D + c] : atL[(size_t)node * D + c];
                if (f < 0) break;
                path.push_back(f);
                node = right ? edges[f].first : edges[f].second;
                right = !right;
                c = (c == a) ? b : a;
            }
            for (int f : path) {
                atL[(size_t)edges[f].first * D + colr[f]] = -1;
                atR[(size_t)edges[f].second * D + colr[f]] = -1;
            }
            for (int f : path) {
                colr[f] = (colr[f] == a) ? b : a;
                atL[(size_t)edges[f].first * D + colr[f]] = f;
                atR[(size_t)edges[f].second * D + colr[f]] = f;
            }
        }
        colr[e] = a;
        atL[(size_t)l * D + a] = e;
        atR[(size_t)r * D + a] = e;
    }
    return colr;
}

}  // namespace

namespace {

// Planned layouts of this process, keyed by the check matrix and the variant
// shape: graphs of one code at several error rates, and the autotuner's
// repeated switches between variants, plan each layout once.  Bounded: the
// cache is emptied when it holds 32 layouts.
struct LayoutKey {
    uint64_t hash;
    int M, N, G, npos, dc;
    bool operator<(const LayoutKey &o) const
    {
        return std::tie(hash, M, N, G, npos, dc) < std::tie(o.hash, o.M, o.N, o.G, o.npos, o.dc);
    }
};

uint64_t fnv1a(const std::vector<int32_t> &a, uint64_t h)
{
    for (int32_t v : a) {
        for (int s = 0; s < 32; s += 8) {
            h ^= (uint64_t)((uint32_t)v >> s) & 0xFFu;
            h *= 0x100000001B3ull;
        }
    }
    return h;
}

void plan_layout_uncached(int M, int N, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col,
                          int G, int npos, int dc, bool optimize, const std::vector<int> &pass_cv, Layout &out);

}  // namespace

void plan_layout(int M, int N, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col, int G,
                 int npos, int dc, bool optimize, const std::vector<int> &pass_cv, Layout &out)
{
    if (!optimize || G % 32 != 0) {
        plan_layout_uncached(M, N, row_ptr, col, G, npos, dc, optimize, pass_cv, out);
        return;
    }
    static std::mutex mu;
    static std::map<LayoutKey, Layout> cache;
    std::vector<int32_t> pcv(pass_cv.begin(), pass_cv.end());
    const LayoutKey key{fnv1a(pcv, fnv1a(col, fnv1a(row_ptr, 0xCBF29CE484222325ull))), M, N, G, npos, dc};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            out = it->second;
            return;
        }
    }
    plan_layout_uncached(M, N, row_ptr, col, G, npos, dc, optimize, pass_cv, out);
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() >= 32) cache.clear();
    cache.emplace(key, out);
}

namespace {

void plan_layout_uncached(int M, int N, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col,
                          int G, int npos, int dc, bool optimize, const std::vector<int> &pass_cv, Layout &out)
{
    out.pos_of_var.assign(N, -1);
    out.var_at_pos.assign(npos, -1);
    out.edge_round.assign(col.size(), 0);
    bool uniform_cv = true;
    for (size_t p = 1; p < pass_cv.size(); ++p) uniform_cv &= pass_cv[p] == pass_cv[0];
    if (!optimize || G % 32 != 0) {
        // identity placement (in order of decreasing degree under a
        // non-uniform slot profile) and CSR edge order
        std::vector<int> order(N);
        std::iota(order.begin(), order.end(), 0);
        if (!uniform_cv) {
            std::vector<int> dg(N, 0);
            for (int32_t c : col) dg[c]++;
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dg[a] > dg[b]; });
        }
        for (int r = 0; r < N; ++r) {
            out.pos_of_var[order[r]] = r;
            out.var_at_pos[r] = order[r];
        }
        for (int i = 0; i < M; ++i)
            for (int a = row_ptr[i], k = 0; a < row_ptr[i + 1]; ++a, ++k) out.edge_round[a] = k;
        return;
    }
    // 1. bank classes, under the per-pass slot counts: a bank's k-th position
    // is k*32 + b, in pass k / (G/32), so a bank may hold (G/32) variables of
    // degree >= d per pass with at least d slots
    std::vector<int> deg(N, 0);
    for (int32_t c : col) deg[c]++;
    std::vector<int> cap_ge;
    const bool uniform = uniform_cv;
    if (!uniform) {
        const int dmax = *std::max_element(deg.begin(), deg.end());
        cap_ge.assign((size_t)dmax + 1, 0);
        for (int d = 0; d <= dmax; ++d)
            for (int p = 0; p < (int)pass_cv.size() && p * G < npos; ++p)
                if (pass_cv[p] >= d) cap_ge[d] += G / 32;
    }
    std::vector<int> bank;
    assign_banks(M, N, row_ptr, col, npos / 32, cap_ge, bank);
    // members of each bank in order of decreasing degree (ties by index) take
    // its positions in order, so higher degrees land in the wider passes
    std::vector<int> order(N);
    std::iota(order.begin(), order.end(), 0);
    if (!uniform) std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return deg[a] > deg[b]; });
    std::vector<int> next(32, 0);   // k-th free position of a bank: k*32 + b
    for (int j : order) {
        const int b = bank[j];
        const int pos = next[b]++ * 32 + b;
        out.pos_of_var[j] = pos;
        out.var_at_pos[pos] = j;
    }
    // 2. edge rounds per group of 32 checks
    for (int g0 = 0; g0 < M; g0 += 32) {
        const int g1 = std::min(M, g0 + 32);
        std::vector<std::pair<int, int>> edges;
        std::vector<int> eid;
        int per_bank[32] = {0};
        std::vector<int> vnode;
        for (int i = g0; i < g1; ++i)
            for (int a = row_ptr[i]; a < row_ptr[i + 1]; ++a) {
                const int b = out.pos_of_var[col[a]] % 32;
                const int virt = per_bank[b]++ / dc;   // split overloaded banks
                edges.emplace_back(i - g0, b * 64 + virt);
                eid.push_back(a);
            }
        // compact right-node ids
        std::vector<int> ids;
        for (auto &e : edges) ids.push_back(e.second);
        std::sort(ids.begin(), ids.end());
        ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
        for (auto &e : edges) e.second = (int)(std::lower_bound(ids.begin(), ids.end(), e.second) - ids.begin());
        const std::vector<int> c = color_group(g1 - g0, (int)ids.size(), dc, edges);
        for (size_t t = 0; t < edges.size(); ++t) out.edge_round[eid[t]] = c[t];
    }
}

}  // namespace

}  // namespace bpdc
