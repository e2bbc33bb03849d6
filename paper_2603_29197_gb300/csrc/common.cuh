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
// max / min of non-negative doubles through their bit patterns (IEEE order of
// non-negative doubles equals the integer order of their bits, +inf included): runs on
// the integer pipe, which on GB300 is far wider than the FP64 pipe
__device__ __forceinline__ double warp_max_nonneg(double v) {
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t > b ? t : b;
    }
    return __longlong_as_double(b);
}
// max of a non-negative accumulator a and |b| through bit patterns, with b's sign bit
// cleared on the integer pipe: a NaN of either sign ends above +inf in that order and
// propagates, where fmax would drop it
__device__ __forceinline__ double amax(double a, double b) {
    const long long bb = __double_as_longlong(b) & 0x7fffffffffffffffLL;
    return bb > __double_as_longlong(a) ? __longlong_as_double(bb) : a;
}
__device__ __forceinline__ double warp_min_nonneg(double v) {
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t < b ? t : b;
    }
    return __longlong_as_double(b);
}

// 1/d by one third-order (Chebyshev) step from the hardware's approximate reciprocal r:
// with e = 1 − d·r, r(1 + e + e²) has relative error e³ (1 − d·r(1+e+e²) = e³ exactly),
// and the seed's e ≲ 2^-22 puts e³ far below the FP64 rounding level.  Three dependent
// FMAs, one fewer than two quadratic Newton steps; every FP64 instruction is scarce on
// this part.  d must be a normal number (pivots are kept away from zero by the dynamic
// regularisation).
__device__ __forceinline__ double recip(double d) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
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

// Block-wide reduction of NV values (sum, or max of non-negative values, per `is_max`),
// result valid in thread 0.  `sm` holds NV * 32 doubles.  All threads must call.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&v)[NV], const bool (&is_max)[NV], double* sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = is_max[k] ? warp_max_nonneg(v[k]) : warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[k * 32 + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < nw ? sm[k * 32 + lane] : 0.0;
            v[k] = is_max[k] ? warp_max_nonneg(t) : warp_sum(t);
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
