// Shared device helpers and the device-side views of the solver's data.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace qoco {

constexpr int kWarp = 32;
// SOC blocks up to this dimension get one thread per cone; larger ones one warp.
constexpr int kSmallCone = 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// sub-warp reductions over aligned groups of G lanes (G a power of two ≤ 32)
template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ double group_max(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide reduction of NV values (sum or max selected per value by `is_max`),
// result valid in thread 0.  `sm` holds NV * 32 doubles.  All threads must call.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], const bool (&is_max)[NV], double* sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = is_max[k] ? warp_max(v[k]) : warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[k * 32 + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < nw ? sm[k * 32 + lane] : (is_max[k] ? 0.0 : 0.0);
            v[k] = is_max[k] ? warp_max(t) : warp_sum(t);
        }
    }
    __syncthreads();
}

}  // namespace qoco

#define QOCO_CUDA_TRY(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) return ::qoco::cuda_fail(_e, #expr, __FILE__, __LINE__); \
    } while (0)

namespace qoco {
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);
}
