// Vector kernels of the GMRES refinement (krylov.h): the FP64 Krylov basis of a solve
// whose factor has FP32 large fronts.  Every reduction is a fixed-order two-stage sum
// (block partials, then one block per result), so repeated solves are bitwise equal.
#include "krylov.h"

namespace qoco {

namespace {

constexpr int kKThreads = 256;
constexpr int kKBlocks = 152 * 4;  // partial sums per dot product

// partial[k·kKBlocks + b] = Σ over block b's grid-stride share of V_k · w, k < nv
__global__ void __launch_bounds__(kKThreads) k_dots(const double* __restrict__ V, int64_t ld, int nv,
                                                    const double* __restrict__ w, int64_t N,
                                                    double* __restrict__ partial) {
    __shared__ double sm[kKThreads / 32];
    const int k = blockIdx.y;
    const double* v = V + (int64_t)k * ld;
    double a = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kKThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kKThreads)
        a = fma(v[i], w[i], a);
    a = warp_sum(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    if (wid == 0) {
        double t = lane < kKThreads / 32 ? sm[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = t;
    }
}

// out[k] (+)= Σ_b partial[k·nb + b], one block per k, fixed order
__global__ void __launch_bounds__(kKThreads) k_dots_finish(const double* __restrict__ partial, int nb,
                                                           double* __restrict__ out, int accumulate) {
    __shared__ double sm[kKThreads / 32];
    const int k = blockIdx.x;
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += kKThreads) a += partial[(int64_t)k * nb + b];
    a = warp_sum(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    if (wid == 0) {
        double t = lane < kKThreads / 32 ? sm[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) out[k] = accumulate ? out[k] + t : t;
    }
}

// w −= Σ_{k < nv} c[k]·V_k
__global__ void k_sub_combination(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ c,
                                  double* __restrict__ w, int64_t N) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double a = w[i];
        for (int k = 0; k < nv; ++k) a = fma(-c[k], V[(int64_t)k * ld + i], a);
        w[i] = a;
    }
}

// u = Σ_{k < nv} c[k]·V_k
__global__ void k_combination(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ c,
                              double* __restrict__ u, int64_t N) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int k = 0; k < nv; ++k) a = fma(c[k], V[(int64_t)k * ld + i], a);
        u[i] = a;
    }
}

// dst = sign·src / √(*nrm2)
__global__ void k_scale_by_norm(const double* __restrict__ src, double* __restrict__ dst, int64_t N,
                                const double* __restrict__ nrm2, double sign) {
    const double s = sign / sqrt(*nrm2);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = s * src[i];
}

// dst = src / den (inverse = false) or src · den (inverse = true), den_i taken as 1 where
// it is not a positive finite number (a row of zeros with a zero right-hand side)
__global__ void k_row_scale(const double* __restrict__ src, const double* __restrict__ den, double* __restrict__ dst,
                            int64_t N, int inverse) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = den[i];
        const double dd = (d > 0.0 && isfinite(d)) ? d : 1.0;
        dst[i] = inverse ? src[i] * dd : src[i] / dd;
    }
}

unsigned vgrid(int64_t N) {
    const int64_t b = (N + 255) / 256;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, kKBlocks));
}

}  // namespace

int krylov_partials() { return kKBlocks * (kKrylovRestart + 2); }

int launch_dots(const double* V, int64_t ld, int nv, const double* w, int64_t N, double* partial, double* out,
                bool accumulate, cudaStream_t st) {
    const unsigned nb = vgrid(N);
    k_dots<<<dim3(nb, nv), kKThreads, 0, st>>>(V, ld, nv, w, N, partial);
    k_dots_finish<<<nv, kKThreads, 0, st>>>(partial, (int)nb, out, accumulate ? 1 : 0);
    return 2;
}

int launch_sub_combination(const double* V, int64_t ld, int nv, const double* c, double* w, int64_t N,
                           cudaStream_t st) {
    k_sub_combination<<<vgrid(N), 256, 0, st>>>(V, ld, nv, c, w, N);
    return 1;
}

int launch_combination(const double* V, int64_t ld, int nv, const double* c, double* u, int64_t N,
                       cudaStream_t st) {
    k_combination<<<vgrid(N), 256, 0, st>>>(V, ld, nv, c, u, N);
    return 1;
}

int launch_scale_by_norm(const double* src, double* dst, int64_t N, const double* nrm2, double sign,
                         cudaStream_t st) {
    k_scale_by_norm<<<vgrid(N), 256, 0, st>>>(src, dst, N, nrm2, sign);
    return 1;
}

int launch_row_scale(const double* src, const double* den, double* dst, int64_t N, bool inverse, cudaStream_t st) {
    k_row_scale<<<vgrid(N), 256, 0, st>>>(src, den, dst, N, inverse ? 1 : 0);
    return 1;
}

}  // namespace qoco
