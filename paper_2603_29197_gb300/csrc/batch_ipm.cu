// The persistent batched kernel's host side and the per-batch summary; the kernel itself
// is batch_ipm.cuh, instantiated per precision in batch_ipm_f64.cu and batch_ipm_mixed.cu
// (two translation units, compiled side by side).
#include "batch_ipm.h"

#include <algorithm>

#include "fronts.cuh"

namespace qoco {

// one instantiation per (warps per CTA, resident warps per SM), see batch_ipm_kernel_*
const void* batch_ipm_kernel_f64(int nw, int dense);
const void* batch_ipm_kernel_mixed(int nw, int dense);

namespace {

// every-instance summary of a batched solve: S.converged = all converged, S.converged_inacc
// = every instance converged or meets the inaccurate tolerances, S.nonfinite = some
// instance met a non-finite value, S.max_iters = the most iterations, S.gap = largest gap
__device__ __forceinline__ double bits_max_s(double a, double b) {
    return __double_as_longlong(b) > __double_as_longlong(a) ? b : a;
}

__global__ void k_batch_summary(BatchView B, IPMScalars* S) {
    __shared__ int sc[32], si[32], sn[32], sm[32];
    __shared__ double sg[32];
    int all = 1, inacc = 1, bad = 0, mit = 0;
    double g = 0.0;
    for (int i = threadIdx.x; i < B.nb; i += blockDim.x) {
        all &= B.conv[i];
        inacc &= B.conv_inacc[i];
        bad |= B.nonfinite[i];
        mit = max(mit, B.iters[i]);
        g = amax(g, B.gap[i]);
    }
    all = __all_sync(0xffffffffu, all);
    inacc = __all_sync(0xffffffffu, inacc);
    bad = __any_sync(0xffffffffu, bad);
    for (int o = 16; o > 0; o >>= 1) mit = max(mit, __shfl_xor_sync(0xffffffffu, mit, o));
    g = warp_max_nonneg(g);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sc[wid] = all; si[wid] = inacc; sn[wid] = bad; sm[wid] = mit; sg[wid] = g; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            all &= sc[w]; inacc &= si[w]; bad |= sn[w]; mit = max(mit, sm[w]); g = bits_max_s(g, sg[w]);
        }
        S->converged = all;
        S->converged_inacc = inacc;
        S->nonfinite = bad;
        S->max_iters = mit;
        S->gap = g;
    }
}

size_t batch_ipm_smem(int nw, int fmax) { return (size_t)nw * wfactor_stride(fmax) * sizeof(double); }

const void* batch_ipm_kernel(int nw, int dense, bool mixed) {
    return mixed ? batch_ipm_kernel_mixed(nw, dense) : batch_ipm_kernel_f64(nw, dense);
}

}  // namespace

int batch_ipm_grid(int nw, int dense, bool mixed, int fmax, int nb, int* grid) {
    const void* k = batch_ipm_kernel(nw, dense, mixed);
    const size_t sm = batch_ipm_smem(nw, fmax);
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int dev = 0, nsm = 0, occ = 0;
    QOCO_CUDA_TRY(cudaGetDevice(&dev));
    QOCO_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    QOCO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, nw * 32, sm));
    *grid = occ < 1 ? 0 : std::min(nb, nsm * occ);
    return 0;
}

int launch_batch_summary(const BatchView& B, IPMScalars* S, cudaStream_t st) {
    k_batch_summary<<<1, 1024, 0, st>>>(B, S);
    return 1;
}

int launch_batch_ipm(const BatchIPMArgs& A, int nw, int dense, int grid, cudaStream_t st) {
    QOCO_CUDA_TRY(cudaMemsetAsync(A.next, 0, sizeof(unsigned int), st));
    const size_t sm = batch_ipm_smem(nw, A.fmax);
    BatchIPMArgs a = A;
    void* args[] = {(void*)&a};
    QOCO_CUDA_TRY(cudaLaunchKernel(batch_ipm_kernel(nw, dense, A.mixed), dim3(grid), dim3(nw * 32), args, sm, st));
    return 1;
}

}  // namespace qoco
