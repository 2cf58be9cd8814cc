// Shared-memory bandwidth microbenchmark: the roof of the decode kernels,
// whose messages live in shared memory and move as one 4-byte load and one
// 4-byte store per message per phase.
//
// Every thread streams 4-byte loads and stores over a conflict-free 64 KB
// tile (lane-consecutive words, like the variable-major message slots), so
// each warp-wide access is one 128-byte wavefront.  Blocks fill every SM in
// one wave; CUDA events around the launch give the bytes moved per second.
#include <cuda_runtime.h>

#include <cstdint>

#include "bpdc_internal.h"

namespace bpdc {
namespace {

constexpr int kPeakThreads = 1024;
constexpr int kPeakWords = 16 * kPeakThreads;   // 64 KB per block

__global__ void __launch_bounds__(kPeakThreads, 2) smem_peak_kernel(int reps, uint32_t *sink)
{
    extern __shared__ uint32_t tile[];   // kPeakWords words
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(tile) + 4u * threadIdx.x;
    for (int i = threadIdx.x; i < kPeakWords; i += blockDim.x) tile[i] = i;
    __syncthreads();
    uint32_t acc = threadIdx.x;
    for (int r = 0; r < reps; ++r) {
        uint32_t v0, v1, v2, v3, v4, v5, v6, v7;
        asm volatile(
            "ld.shared.b32 %0, [%8];\n\t"
            "ld.shared.b32 %1, [%8+4096];\n\t"
            "ld.shared.b32 %2, [%8+8192];\n\t"
            "ld.shared.b32 %3, [%8+12288];\n\t"
            "ld.shared.b32 %4, [%8+16384];\n\t"
            "ld.shared.b32 %5, [%8+20480];\n\t"
            "ld.shared.b32 %6, [%8+24576];\n\t"
            "ld.shared.b32 %7, [%8+28672];"
            : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3), "=r"(v4), "=r"(v5), "=r"(v6), "=r"(v7)
            : "r"(base));
        acc ^= v0 ^ v1 ^ v2 ^ v3 ^ v4 ^ v5 ^ v6 ^ v7;
        asm volatile(
            "st.shared.b32 [%0+32768], %1;\n\t"
            "st.shared.b32 [%0+36864], %2;\n\t"
            "st.shared.b32 [%0+40960], %3;\n\t"
            "st.shared.b32 [%0+45056], %4;\n\t"
            "st.shared.b32 [%0+49152], %5;\n\t"
            "st.shared.b32 [%0+53248], %6;\n\t"
            "st.shared.b32 [%0+57344], %7;\n\t"
            "st.shared.b32 [%0+61440], %8;"
            ::"r"(base), "r"(acc), "r"(v0), "r"(v1), "r"(v2), "r"(v3), "r"(v4), "r"(v5), "r"(v6)
            : "memory");
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;   // keeps the loop observable
}

}  // namespace

cudaError_t measure_smem_peak(int reps, double *bytes_per_s, int *num_sms)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int smem = kPeakWords * 4;
    e = cudaFuncSetAttribute((const void *)smem_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)smem_peak_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_peak_kernel, kPeakThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int grid = per_sm * sms;   // one full wave: every block of an SM runs concurrently
    uint32_t *sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&sink, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    double best_bps = 0.0;
    for (int trial = 0; e == cudaSuccess && trial < 4; ++trial) {
        const int r = trial == 0 ? reps / 8 : reps;   // the first run warms up
        e = cudaEventRecord(a, 0);
        if (e == cudaSuccess) {
            smem_peak_kernel<<<grid, kPeakThreads, smem>>>(r, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess || trial == 0 || ms <= 0.0f) continue;
        const double bytes = 64.0 * kPeakThreads * (double)r * grid;   // 8 loads + 8 stores of 4 B
        const double bps = bytes / (ms * 1e-3);
        if (bps > best_bps) best_bps = bps;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return e;
    *bytes_per_s = best_bps;
    *num_sms = sms;
    return cudaSuccess;
}

}  // namespace bpdc
