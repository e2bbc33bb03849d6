// FP64 throughput of this GPU, measured by the library's own kernels: the FP64 work of
// the factorisation (paper §2.2: the numeric LDLᵀ of eq. (2)) runs either on the FP64
// FMA units (DFMA) or, for a contraction, could run on the FP64 tensor-core path
// (mma.sync m8n8k4 f64, "DMMA").  These two rates are the denominators of the FP64
// rooflines, so they are measured here rather than taken from a data sheet.
//
// Both kernels issue long runs of independent operations from every warp of a grid of
// blocks resident on every SM; the time of one launch (CUDA events on the caller's
// stream, best of several launches) gives flops/s.  Results are written to global
// memory only under a condition the inputs never meet, so no work is optimised away.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "qoco_gpu.h"

namespace qoco {
namespace {

constexpr int kPeakIters = 4096;

// 8 independent FMA chains per thread: a·x + b with a close to 1 (no overflow)
__global__ void __launch_bounds__(256) k_peak_dfma(double a, double b, double* sink) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = threadIdx.x * 1e-3 + u;
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = fma(a, x[u], b);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
    if (s == -1.2345) sink[blockIdx.x] = s;
}

// 4 independent accumulator tiles per warp: D = A·B + D, m8n8k4, FP64 in and out
__global__ void __launch_bounds__(256) k_peak_dmma(double av, double bv, double* sink) {
    const double a = av + (threadIdx.x & 31) * 1e-9, b = bv;
    double d[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) d[u][0] = d[u][1] = 0.0;
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(d[u][0]), "+d"(d[u][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) s += d[u][0] + d[u][1];
    if (s == -1.2345) sink[blockIdx.x] = s;
}

template <class K>
int time_kernel(K kern, int blocks, double* sink, cudaStream_t st, float* best_ms) {
    cudaEvent_t e0, e1;
    QOCO_CUDA_TRY(cudaEventCreate(&e0));
    QOCO_CUDA_TRY(cudaEventCreate(&e1));
    *best_ms = 0.0f;
    int rc = 0;
    for (int rep = 0; rep < 6 && !rc; ++rep) {
        cudaError_t e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            kern<<<blocks, 256, 0, st>>>(0.999999, 1e-7, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) rc = cuda_fail(e, "peak kernel", __FILE__, __LINE__);
        else if (rep > 0 && (*best_ms == 0.0f || ms < *best_ms)) *best_ms = ms;  // launch 0 warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace
}  // namespace qoco

using namespace qoco;

extern "C" int qoco_gpu_fp64_peaks(double* dfma_gflops, double* dmma_gflops, void* stream) {
    if (!dfma_gflops || !dmma_gflops) return QOCO_GPU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    QOCO_CUDA_TRY(cudaGetDevice(&dev));
    QOCO_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = 8 * nsm;  // 64 warps per SM
    double* sink = nullptr;
    QOCO_CUDA_TRY(cudaMalloc((void**)&sink, sizeof(double) * blocks));
    float ms_f = 0.0f, ms_m = 0.0f;
    int rc = time_kernel(k_peak_dfma, blocks, sink, st, &ms_f);
    if (!rc) rc = time_kernel(k_peak_dmma, blocks, sink, st, &ms_m);
    cudaFree(sink);
    if (rc) return rc;
    const double threads = (double)blocks * 256.0, warps = threads / 32.0;
    const double f_dfma = threads * kPeakIters * 8 * 2.0;             // 2 flops per FMA
    const double f_dmma = warps * kPeakIters * 4 * (2.0 * 8 * 8 * 4);  // 512 flops per m8n8k4
    *dfma_gflops = ms_f > 0.0f ? f_dfma / (ms_f * 1e-3) / 1e9 : 0.0;
    *dmma_gflops = ms_m > 0.0f ? f_dmma / (ms_m * 1e-3) / 1e9 : 0.0;
    return 0;
}
