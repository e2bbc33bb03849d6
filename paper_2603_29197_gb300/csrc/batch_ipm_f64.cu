// The persistent batched kernel (batch_ipm.cuh) with FP64 fronts: one instantiation per
// warps per CTA (1, 2, 4) and resident warps per SM asked of the compiler (16 or 32).
#include "batch_ipm.cuh"

namespace qoco {

const void* batch_ipm_kernel_f64(int nw, int dense) {
    using namespace batch_ipm_detail;
    constexpr bool M = false;
    if (nw == 1) return dense ? (const void*)k_batch_ipm<1, 32, M> : (const void*)k_batch_ipm<1, 16, M>;
    if (nw == 2) return dense ? (const void*)k_batch_ipm<2, 16, M> : (const void*)k_batch_ipm<2, 8, M>;
    return dense ? (const void*)k_batch_ipm<4, 8, M> : (const void*)k_batch_ipm<4, 4, M>;
}

}  // namespace qoco
