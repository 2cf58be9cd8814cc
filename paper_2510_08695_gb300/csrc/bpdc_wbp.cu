// Weighted product-sum BP with a hand-written adjoint (differentiable
// decoding; not part of the paper).  For iterations t = 0..T-1 over the edges
// e = (i, j) of H in CSR order, with weights W[0][t][e] (check -> variable,
// wc) and W[1][t][e] (variable -> check, wv):
//
//   q_e(t) = clip(wv[t][e] * (lambda_j + sum_{e' in M(j), e' != e} r_e'(t-1)), -Q, Q),   r(-1) = 0
//   r_e(t) = wc[t][e] * (-1)^{s_i} prod_{e' in N(i), e' != e} sgn(q_e'(t))
//                     * phi(sum_{e' in N(i), e' != e} phi(max(|q_e'(t)|, qmin)))
//   L_j(t) = lambda_j + sum_{e in M(j)} r_e(t)
//
// phi(x) = -log tanh(x/2) (Sec. II.C.1's product-sum rule in log form).  With
// unit weights and no clipping this is the decoder's flooding product-sum BP.
//
// Forward: one warp per shot, q and r of the shot in shared memory; the q of
// every k-th iteration is checkpointed to global memory.  Adjoint: per shot,
// segments of k iterations are recomputed from their checkpoint into shared
// memory and then run backwards; with phi'(x) = -1/sinh(x),
//   d r_e / d q_e' = wc_e s_e sgn(q_e') / (sinh(S_e) sinh(|q_e'|)),
// so the adjoint of q_e' is sgn(q_e') / sinh(|q_e'|) times the sum over the
// other edges e of the check of rbar_e wc_e s_e / sinh(S_e) (prefix and suffix
// sums, no subtraction).  Every shot writes its own gradient partials; a
// second kernel sums them over shots in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <cstdint>

#include "bpdc_internal.h"

namespace bpdc {
namespace {

constexpr float kQmin = 1e-6f;

__device__ __forceinline__ float wphi(float x) { return log1pf(2.0f / expm1f(x)); }

// 1 / sinh(x) for x > 0 without overflow: 2 e^-x / (1 - e^-2x)
__device__ __forceinline__ float inv_sinh(float x) { return 2.0f * expf(-x) / -expm1f(-2.0f * x); }

__device__ __forceinline__ uint32_t syn_bit(const uint32_t *sy, int i) { return (__ldg(sy + (i >> 5)) >> (i & 31)) & 1u; }

// q(t) from r(t-1): lanes over variables
__device__ void wbp_var_phase(const DevGraph &g, const float *r, float *q, const float *wv, float clip, int lane)
{
    for (int j = lane; j < g.N; j += 32) {
        const int c0 = __ldg(g.c_ptr + j), d = __ldg(g.c_ptr + j + 1) - c0;
        const float lam = __ldg(g.lam_col + j);
        int ee[kWbpMaxCol];
        float rr[kWbpMaxCol], pre[kWbpMaxCol + 1];
        pre[0] = 0.0f;
#pragma unroll
        for (int m = 0; m < kWbpMaxCol; ++m) {
            ee[m] = m < d ? __ldg(g.c_edge + c0 + m) : 0;
            rr[m] = m < d ? r[ee[m]] : 0.0f;
            pre[m + 1] = pre[m] + rr[m];
        }
        float suf = 0.0f;
#pragma unroll
        for (int m = kWbpMaxCol - 1; m >= 0; --m) {
            if (m < d) {
                const float z = __ldg(wv + ee[m]) * (lam + (pre[m] + suf));
                q[ee[m]] = fminf(fmaxf(z, -clip), clip);
                suf += rr[m];
            }
        }
    }
}

// r(t) from q(t): lanes over checks
__device__ void wbp_chk_phase(const DevGraph &g, const float *q, float *r, const float *wc, const uint32_t *sy,
                              int lane)
{
    for (int i = lane; i < g.M; i += 32) {
        const int e0 = __ldg(g.h_ptr + i), d = __ldg(g.h_ptr + i + 1) - e0;
        float f[kWbpMaxRow], suf[kWbpMaxRow + 1];
        uint32_t negs = 0, par = syn_bit(sy, i);
#pragma unroll
        for (int k = 0; k < kWbpMaxRow; ++k) {
            f[k] = 0.0f;
            if (k < d) {
                const float x = q[e0 + k];
                f[k] = wphi(fmaxf(fabsf(x), kQmin));
                const uint32_t ng = x < 0.0f ? 1u : 0u;
                negs |= ng << k;
                par ^= ng;
            }
        }
        suf[kWbpMaxRow] = 0.0f;
#pragma unroll
        for (int k = kWbpMaxRow - 1; k >= 0; --k) suf[k] = suf[k + 1] + f[k];
        float pre = 0.0f;
#pragma unroll
        for (int k = 0; k < kWbpMaxRow; ++k) {
            if (k < d) {
                const float c = wphi(pre + suf[k + 1]);
                const bool neg = ((par ^ (negs >> k)) & 1u) != 0;
                r[e0 + k] = __ldg(wc + e0 + k) * (neg ? -c : c);
                pre += f[k];
            }
        }
    }
}

__global__ void wbp_forward_kernel(DevGraph g, WbpArgs a)
{
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int E = a.E;
    float *r = sm + (size_t)warp * 2 * E, *q = r + E;
    const int nseg = (a.T + a.k - 1) / a.k;
    for (int64_t b = (int64_t)blockIdx.x * wpb + warp; b < a.B; b += (int64_t)gridDim.x * wpb) {
        const uint32_t *sy = a.syn + b * g.MW;
        for (int e = lane; e < E; e += 32) r[e] = 0.0f;
        __syncwarp();
        for (int t = 0; t < a.T; ++t) {
            wbp_var_phase(g, r, q, a.W + (size_t)(a.T + t) * E, a.clip, lane);
            __syncwarp();
            if (a.ckpt && t % a.k == 0) {
                float *ck = a.ckpt + ((size_t)b * nseg + t / a.k) * E;
                for (int e = lane; e < E; e += 32) ck[e] = q[e];
            }
            wbp_chk_phase(g, q, r, a.W + (size_t)t * E, sy, lane);
            __syncwarp();
            if (a.post) {
                float *pr = a.post + ((size_t)b * a.T + t) * g.N;
                for (int j = lane; j < g.N; j += 32) {
                    const int c0 = __ldg(g.c_ptr + j), c1 = __ldg(g.c_ptr + j + 1);
                    float L = __ldg(g.lam_col + j);
                    for (int c = c0; c < c1; ++c) L += r[__ldg(g.c_edge + c)];
                    pr[j] = L;
                }
            }
        }
        __syncwarp();
    }
}

__global__ void wbp_backward_kernel(DevGraph g, WbpArgs a)
{
    extern __shared__ float sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int E = a.E, T = a.T, K = a.k;
    float *Qs = sm + (size_t)warp * (2 * K + 2) * E;   // q(t0 .. t0+K-1) of the current segment
    float *Rs = Qs + (size_t)K * E;                     // r(t0 .. t0+K-1)
    float *QB = Rs + (size_t)K * E;                     // adjoint of q(t+1), then of q(t)
    float *RB = QB + E;                                 // adjoint of r(t)
    const int nseg = (T + K - 1) / K;
    const float clip = a.clip;
    for (int64_t b = (int64_t)blockIdx.x * wpb + warp; b < a.B; b += (int64_t)gridDim.x * wpb) {
        const uint32_t *sy = a.syn + b * g.MW;
        const float *gp = a.gpost + (size_t)b * T * g.N;
        float *part = a.part + (size_t)b * 2 * T * E;   // [2][T][E] partials of this shot
        for (int e = lane; e < E; e += 32) QB[e] = 0.0f;
        for (int seg = nseg - 1; seg >= 0; --seg) {
            const int t0 = seg * K, nt = min(K, T - t0);
            const float *ck = a.ckpt + ((size_t)b * nseg + seg) * E;
            for (int e = lane; e < E; e += 32) Qs[e] = ck[e];
            __syncwarp();
            for (int u = 0; u < nt; ++u) {   // recompute the segment
                wbp_chk_phase(g, Qs + (size_t)u * E, Rs + (size_t)u * E, a.W + (size_t)(t0 + u) * E, sy, lane);
                __syncwarp();
                if (u + 1 < nt) {
                    wbp_var_phase(g, Rs + (size_t)u * E, Qs + (size_t)(u + 1) * E, a.W + (size_t)(T + t0 + u + 1) * E,
                                  clip, lane);
                    __syncwarp();
                }
            }
            for (int u = nt - 1; u >= 0; --u) {
                const int t = t0 + u;
                const float *rt = Rs + (size_t)u * E;
                const float *qt = Qs + (size_t)u * E;
                // (1) adjoint of r(t): posterior L(t) and, through q(t+1), the
                // variable updates of iteration t+1 (also their wv gradient)
                const bool next = t + 1 < T;
                const float *wv1 = a.W + (size_t)(T + t + 1) * E;
                for (int j = lane; j < g.N; j += 32) {
                    const int c0 = __ldg(g.c_ptr + j), d = __ldg(g.c_ptr + j + 1) - c0;
                    const float lam = __ldg(g.lam_col + j);
                    const float gl = gp[(size_t)t * g.N + j];
                    int ee[kWbpMaxCol];
                    float rr[kWbpMaxCol], ab[kWbpMaxCol], pre[kWbpMaxCol + 1];
                    pre[0] = 0.0f;
#pragma unroll
                    for (int m = 0; m < kWbpMaxCol; ++m) {
                        ee[m] = m < d ? __ldg(g.c_edge + c0 + m) : 0;
                        rr[m] = m < d ? rt[ee[m]] : 0.0f;
                        pre[m + 1] = pre[m] + rr[m];
                    }
                    float suf = 0.0f;
#pragma unroll
                    for (int m = kWbpMaxCol - 1; m >= 0; --m) {
                        ab[m] = 0.0f;
                        if (m < d && next) {
                            const float av = lam + (pre[m] + suf);
                            const float w = __ldg(wv1 + ee[m]);
                            const bool in = fabsf(w * av) <= clip;
                            const float qb = QB[ee[m]];
                            ab[m] = in ? qb * w : 0.0f;
                            part[(size_t)(T + t + 1) * E + ee[m]] = in ? qb * av : 0.0f;
                        }
                        if (m < d) suf += rr[m];
                    }
                    float apre[kWbpMaxCol + 1];
                    apre[0] = 0.0f;
#pragma unroll
                    for (int m = 0; m < kWbpMaxCol; ++m) apre[m + 1] = apre[m] + ab[m];
                    float asuf = 0.0f;
#pragma unroll
                    for (int m = kWbpMaxCol - 1; m >= 0; --m) {
                        if (m < d) {
                            RB[ee[m]] = gl + (apre[m] + asuf);
                            asuf += ab[m];
                        }
                    }
                }
                __syncwarp();
                // (2) the check update of iteration t: wc gradient and adjoint of q(t)
                const float *wc = a.W + (size_t)t * E;
                for (int i = lane; i < g.M; i += 32) {
                    const int e0 = __ldg(g.h_ptr + i), d = __ldg(g.h_ptr + i + 1) - e0;
                    float f[kWbpMaxRow], suf[kWbpMaxRow + 1], gk[kWbpMaxRow];
                    uint32_t negs = 0, par = syn_bit(sy, i);
#pragma unroll
                    for (int k = 0; k < kWbpMaxRow; ++k) {
                        f[k] = 0.0f;
                        if (k < d) {
                            const float x = qt[e0 + k];
                            f[k] = wphi(fmaxf(fabsf(x), kQmin));
                            const uint32_t ng = x < 0.0f ? 1u : 0u;
                            negs |= ng << k;
                            par ^= ng;
                        }
                    }
                    suf[kWbpMaxRow] = 0.0f;
#pragma unroll
                    for (int k = kWbpMaxRow - 1; k >= 0; --k) suf[k] = suf[k + 1] + f[k];
                    float pre = 0.0f;
#pragma unroll
                    for (int k = 0; k < kWbpMaxRow; ++k) {
                        gk[k] = 0.0f;
                        if (k < d) {
                            const float S = pre + suf[k + 1];
                            const float s = ((par ^ (negs >> k)) & 1u) ? -1.0f : 1.0f;
                            const float rb = RB[e0 + k];
                            part[(size_t)t * E + e0 + k] = rb * s * wphi(S);
                            gk[k] = rb * __ldg(wc + e0 + k) * s * inv_sinh(S);
                            pre += f[k];
                        }
                    }
                    float gpre[kWbpMaxRow + 1];
                    gpre[0] = 0.0f;
#pragma unroll
                    for (int k = 0; k < kWbpMaxRow; ++k) gpre[k + 1] = gpre[k] + gk[k];
                    float gsuf = 0.0f;
#pragma unroll
                    for (int k = kWbpMaxRow - 1; k >= 0; --k) {
                        if (k < d) {
                            const float x = qt[e0 + k];
                            const float ax = fabsf(x);
                            const float dq = ax >= kQmin ? (x < 0.0f ? -inv_sinh(ax) : inv_sinh(ax)) : 0.0f;
                            QB[e0 + k] = dq * (gpre[k] + gsuf);
                            gsuf += gk[k];
                        }
                    }
                }
                __syncwarp();
            }
        }
        // q(0) = clip(wv[0] lambda): gradient of wv[0]
        for (int j = lane; j < g.N; j += 32) {
            const int c0 = __ldg(g.c_ptr + j), c1 = __ldg(g.c_ptr + j + 1);
            const float lam = __ldg(g.lam_col + j);
            for (int c = c0; c < c1; ++c) {
                const int e = __ldg(g.c_edge + c);
                const float w = __ldg(a.W + (size_t)T * E + e);
                part[(size_t)T * E + e] = fabsf(w * lam) <= clip ? QB[e] * lam : 0.0f;
            }
        }
        __syncwarp();
    }
}

// out[w] = sum over shots b of part[b][w], in shot order, accumulated in FP64
__global__ void wbp_reduce_kernel(const float *part, int64_t B, int64_t n, float *out)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t b = 0; b < B; ++b) s += (double)part[b * n + w];
        out[w] = (float)s;
    }
}

}  // namespace

size_t wbp_smem_forward(int E, int warps) { return (size_t)warps * 2 * E * sizeof(float); }
size_t wbp_smem_backward(int E, int k, int warps) { return (size_t)warps * (2 * k + 2) * E * sizeof(float); }

cudaError_t launch_wbp_forward(const DevGraph &g, const WbpArgs &a, cudaStream_t s)
{
    if (a.B <= 0) return cudaSuccess;
    const int warps = 8;
    const size_t smem = wbp_smem_forward(a.E, warps);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void *)wbp_forward_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (a.B + warps - 1) / warps;
    const int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
    wbp_forward_kernel<<<grid, warps * 32, smem, s>>>(g, a);
    return cudaGetLastError();
}

cudaError_t launch_wbp_backward(const DevGraph &g, const WbpArgs &a, float *grad_w, cudaStream_t s)
{
    const int64_t n = (int64_t)2 * a.T * a.E;
    if (a.B > 0) {
        int warps = 4;
        while (warps > 1 && wbp_smem_backward(a.E, a.k, warps) > kMaxWbpSmem) warps /= 2;
        const size_t smem = wbp_smem_backward(a.E, a.k, warps);
        cudaError_t e = cudaFuncSetAttribute((const void *)wbp_backward_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int64_t blocks = (a.B + warps - 1) / warps;
        const int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
        wbp_backward_kernel<<<grid, warps * 32, smem, s>>>(g, a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int rgrid = (int)((n + 255) / 256);
        wbp_reduce_kernel<<<rgrid, 256, 0, s>>>(a.part, a.B, n, grad_w);
        return cudaGetLastError();
    }
    return cudaMemsetAsync(grad_w, 0, sizeof(float) * n, s);
}

}  // namespace bpdc
