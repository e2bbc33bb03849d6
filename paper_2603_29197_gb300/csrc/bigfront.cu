// Large fronts (paper §2.2: the numeric LDLᵀ of the KKT matrix, eq. (2)), factored and
// solved by sequences of grid-wide kernels instead of one CTA per front.
//
// A front of order f with c pivot columns is a dense f×f column-major block.  The
// partial LDLᵀ runs in panels of nb ≤ kBigNB columns (right-looking):
//   diag     LDLᵀ of the nb×nb diagonal block in shared memory (one CTA)
//   l21      rows below the panel: w = a·L11⁻ᵀ (forward substitution, one thread per
//            row), l = w·D⁻¹; w is kept row-major for the update
//   trailing A22 −= L21·Wᵀ on the lower triangle, 64×64 tiles over the whole GPU
// after which the trailing (f−c)×(f−c) block is the update matrix for the parent.
// The working front is FP64, or FP32 in mixed precision (the factor is then rounded to
// FP32 accuracy; the solves stay FP64 and iterative refinement against the FP64 KKT
// matrix recovers the accuracy).  Children's update blocks are added column by column:
// one warp owns a parent column and walks the children in order, so the sums are
// deterministic without atomics.
//
// The solves of a large front are blocked the same way: per panel block one launch
// in which every CTA solves the nb×nb triangle redundantly (a short dependent chain)
// and then updates its own rows, so no second launch or grid barrier is needed.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "factor.h"

namespace qoco {

namespace {

constexpr int kBT = 64;  // trailing-update tile (rows and columns)

template <class T>
__device__ __forceinline__ T rcp_t(T d);
template <>
__device__ __forceinline__ double rcp_t<double>(double d) { return recip(d); }
template <>
__device__ __forceinline__ float rcp_t<float>(float d) { return 1.0f / d; }

template <class T>
__global__ void k_big_zero(T* __restrict__ F, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        F[i] = T(0);
}

// KKT entries of the front (with the static regularisation on its pivot diagonal)
template <class T>
__global__ void k_big_assemble(int s, FactorView a, const double* __restrict__ kval, T* __restrict__ F) {
    const int f = a.nrow[s], first = a.first[s];
    const int64_t e0 = a.amap_ptr[s], e1 = a.amap_ptr[s + 1];
    for (int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e1;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int off = a.amap_off[e];
        double v = kval[a.amap_slot[e]];
        const int col = off / f, row = off - col * f;
        if (row == col) v += a.dsign[first + col] > 0 ? a.eps : -a.eps;
        F[off] = (T)v;
    }
}

// extend-add of every child's update block; one warp per parent column j walks the
// child columns that land on j (precomputed list, child order) and adds them
template <class T>
__global__ void k_big_extend_add(int s, FactorView a, const int64_t* __restrict__ ea_ptr,
                                 const int* __restrict__ ea_child, const int* __restrict__ ea_pos, T* __restrict__ F) {
    const int f = a.nrow[s];
    const int lane = threadIdx.x & 31;
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (j >= f) return;
    T* Fj = F + (int64_t)j * f;
    for (int64_t e = ea_ptr[j]; e < ea_ptr[j + 1]; ++e) {
        const ChildInfo ci = a.cinfo[ea_child[e]];
        const int jj = ea_pos[e];
        const int* rel = a.rel + ci.rel_off;
        const double* U = a.front + ci.u_off + (int64_t)jj * ci.fc;
        for (int ii = jj + lane; ii < ci.r; ii += 32) Fj[rel[ii]] += (T)U[ii];
    }
}

// LDLᵀ of the nb×nb diagonal block at (k0, k0); one CTA.  Columns stay unscaled until
// the end, and the thread that owns the next diagonal entry computes the next pivot as
// soon as it has applied the current column to it, so each column costs one barrier.
// Entry (i, j) of the lower triangle belongs to thread (i·(i+1)/2 + j) mod blockDim.
template <class T>
__global__ void __launch_bounds__(256) k_big_diag(int s, int k0, int nb, FactorView a, T* __restrict__ F,
                                                  double* __restrict__ Xinv) {
    constexpr int kOwn = (kBigNB * (kBigNB + 1) / 2 + 255) / 256;  // entries per thread
    __shared__ T D[kBigNB][kBigNB + 1];
    __shared__ T s_inv[kBigNB];
    const int f = a.nrow[s], first = a.first[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ntri = nb * (nb + 1) / 2;
    for (int t = tid; t < nb * nb; t += nt) {
        const int j = t / nb, i = t - j * nb;
        if (i >= j) D[i][j] = F[(int64_t)(k0 + j) * f + k0 + i];
    }
    // this thread's entries (i, j) of the lower triangle, i ≥ j, in a fixed order
    int oi[kOwn], oj[kOwn];
#pragma unroll
    for (int u = 0; u < kOwn; ++u) {
        const int t = tid + u * 256;
        if (t < ntri) {
            int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
            while ((i + 1) * (i + 2) / 2 <= t) ++i;
            while (i * (i + 1) / 2 > t) --i;
            oi[u] = i;
            oj[u] = t - i * (i + 1) / 2;
        } else {
            oi[u] = -1;
            oj[u] = kBigNB;
        }
    }
    __syncthreads();
    int nreg = 0;
    auto pivot = [&](int k) {
        double d = (double)D[k][k];
        const bool pos = a.dsign[first + k0 + k] > 0;
        const bool ok = pos ? (d >= a.dyn_thresh) : (d <= -a.dyn_thresh);
        if (!ok) { d = pos ? a.dyn_value : -a.dyn_value; ++nreg; }
        const T dt = (T)d;
        D[k][k] = dt;
        s_inv[k] = rcp_t<T>(dt);
    };
    if (tid == 0) pivot(0);
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        const T inv = s_inv[k];
#pragma unroll
        for (int u = 0; u < kOwn; ++u) {
            const int i = oi[u], j = oj[u];
            if (j <= k) continue;
            D[i][j] -= D[i][k] * D[j][k] * inv;
            if (i == k + 1 && j == k + 1) pivot(k + 1);
        }
        __syncthreads();
    }
    // FP64 reciprocal pivots for the solves (off the pivot chain)
    for (int k = tid; k < nb; k += nt) a.dinv[first + k0 + k] = recip((double)D[k][k]);
    // L (scaled columns) and D back to the front; the strictly lower part of D becomes L
    for (int t = tid; t < nb * nb; t += nt) {
        const int j = t / nb, i = t - j * nb;
        if (i > j) {
            const T l = D[i][j] * s_inv[j];
            F[(int64_t)(k0 + j) * f + k0 + i] = l;
            D[i][j] = l;
        } else if (i == j) {
            F[(int64_t)(k0 + j) * f + k0 + i] = D[i][j];
        }
    }
    __syncthreads();
    // in-place inverse of the unit lower triangle (in the working precision): after step
    // k, rows ≤ k hold L⁻¹'s rows; row i > k takes X_ij ← X_ij − L_ik·X_kj for j < k and
    // X_ik ← −L_ik (L_ik is read from column k before that column is overwritten)
    for (int k = 0; k < nb - 1; ++k) {
        const int m = nb - 1 - k;  // rows k+1 .. nb−1
        for (int t = tid; t < m * k; t += nt) {
            const int ii = t / k, j = t - ii * k;
            const int i = k + 1 + ii;
            D[i][j] -= D[i][k] * D[k][j];
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < nb; i += nt) D[i][k] = -D[i][k];
        __syncthreads();
    }
    // store row-major: Xinv[i·kBigNB + j] = (L_bb⁻¹)_ij (unit diagonal, zero above)
    for (int t = tid; t < nb * nb; t += nt) {
        const int i = t / nb, j = t - i * nb;
        Xinv[i * kBigNB + j] = j < i ? (double)D[i][j] : (j == i ? 1.0 : 0.0);
    }
    if (nreg) atomicAdd(a.nreg, nreg);
}

// rows i ≥ k0+nb: w = a_i· L11⁻ᵀ, l_i· = w D⁻¹ (into F), w into W[i·kBigNB + k]
template <class T>
__global__ void __launch_bounds__(128) k_big_l21(int s, int k0, int nb, FactorView a, T* __restrict__ F,
                                                 T* __restrict__ W) {
    __shared__ T L11[kBigNB][kBigNB + 1];
    __shared__ T dv[kBigNB];
    const int f = a.nrow[s], first = a.first[s];
    for (int t = threadIdx.x; t < kBigNB * kBigNB; t += blockDim.x) {
        const int j = t / kBigNB, i = t - j * kBigNB;
        L11[i][j] = (i > j && i < nb) ? F[(int64_t)(k0 + j) * f + k0 + i] : T(0);
    }
    for (int k = threadIdx.x; k < nb; k += blockDim.x) dv[k] = (T)a.dinv[first + k0 + k];
    __syncthreads();
    const int i = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f) return;
    T* wr = W + (int64_t)i * kBigNB;
    // two halves of 32 columns keep the row in registers without spills: the second
    // half first takes the first half's contribution (re-read from W, written by this
    // same thread), then both halves run the forward substitution with their diagonal
    // block of L11
    for (int kb = 0; kb < nb; kb += 32) {
        T w[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) w[k] = kb + k < nb ? F[(int64_t)(k0 + kb + k) * f + i] : T(0);
        for (int j = 0; j < kb; ++j) {
            const T wj = wr[j];
#pragma unroll
            for (int k = 0; k < 32; ++k) w[k] -= wj * L11[kb + k][j];
        }
#pragma unroll
        for (int k = 1; k < 32; ++k) {
            T acc = w[k];
#pragma unroll
            for (int j = 0; j < k; ++j) acc -= w[j] * L11[kb + k][kb + j];
            w[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (kb + k < nb) {
                wr[kb + k] = w[k];
                F[(int64_t)(k0 + kb + k) * f + i] = w[k] * dv[kb + k];
            }
    }
}

// A22 −= L21·Wᵀ on the lower triangle of rows/columns [base, f); one CTA per 64×64
// tile of the lower triangle (tile index → (ti, tj), ti ≥ tj), 256 threads, 4×4 each
template <class T>
__global__ void __launch_bounds__(256) k_big_trailing(int s, int k0, int nb, FactorView a, T* __restrict__ F,
                                                      const T* __restrict__ W) {
    constexpr int KC = 32;  // panel columns staged per step (keeps the tiles ≤ 33 KB)
    __shared__ T Ls[KC][kBT + 1];
    __shared__ T Ws[KC][kBT + 1];
    const int f = a.nrow[s];
    const int base = k0 + nb;
    // triangular tile index
    const int t = blockIdx.x;
    int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int r0 = base + ti * kBT, c0 = base + tj * kBT;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    for (int kc = 0; kc < nb; kc += KC) {
        const int kn = min(KC, nb - kc);
        for (int e = tid; e < kn * kBT; e += 256) {
            const int k = e / kBT, r = e - k * kBT;
            Ls[k][r] = r0 + r < f ? F[(int64_t)(k0 + kc + k) * f + r0 + r] : T(0);
        }
        for (int e = tid; e < kn * kBT; e += 256) {
            const int cc = e / kn, k = e - cc * kn;
            Ws[k][cc] = c0 + cc < f ? W[(int64_t)(c0 + cc) * kBigNB + kc + k] : T(0);
        }
        __syncthreads();
        for (int k = 0; k < kn; ++k) {
            T lr[4], wc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) lr[u] = Ls[k][tx + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) wc[v] = Ws[k][ty * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += lr[u] * wc[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int j = c0 + ty * 4 + v;
        if (j >= f) continue;
        T* Fj = F + (int64_t)j * f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = r0 + tx + 16 * u;
            if (i < f && i >= j) Fj[i] -= acc[u][v];
        }
    }
}

// FP32 working front → the FP64 front storage (lower triangle)
__global__ void k_big_writeback(const float* __restrict__ Fw, double* __restrict__ G, int f) {
    const int64_t n = (int64_t)f * f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / f), i = (int)(e - (int64_t)j * f);
        if (i >= j) G[e] = (double)Fw[e];
    }
}

// ---- solves ------------------------------------------------------------------------
// forward gather: v = rhs on the pivot rows, 0 below, plus the children's update
// vectors; one thread per row sums the child entries that land on it, in child order
__global__ void k_big_fwd_gather(int s, FactorView a, const int64_t* __restrict__ ea_ptr,
                                 const int* __restrict__ ea_child, const int* __restrict__ ea_pos,
                                 const double* __restrict__ rhs, double* __restrict__ v) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < f; i += gridDim.x * blockDim.x) {
        double acc = i < c ? rhs[a.perm[first + i]] : 0.0;
        for (int64_t e = ea_ptr[i]; e < ea_ptr[i + 1]; ++e) acc += a.upd[a.cinfo[ea_child[e]].rel_off + ea_pos[e]];
        v[i] = acc;
    }
}

// one forward block: y_b = L_bb⁻¹ v_b with the inverse stored by the factorisation
// (every CTA, redundantly: a 64×64 matrix-vector product, no dependent chain), CTA 0
// stores y_b; each CTA updates its rows i ≥ k0+nb: v_i −= Σ_k L_{i,k0+k} y_k
__global__ void __launch_bounds__(256) k_big_fwd_step(int s, int k0, int nb, FactorView a,
                                                      const double* __restrict__ Xb, double* __restrict__ v,
                                                      double* __restrict__ y) {
    __shared__ double vb[kBigNB], yb[kBigNB];
    const int f = a.nrow[s];
    const double* L = a.front + a.front_off[s];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k = tid; k < nb; k += blockDim.x) vb[k] = v[k0 + k];
    __syncthreads();
    for (int i = wid; i < nb; i += blockDim.x >> 5) {
        const double* xr = Xb + i * kBigNB;
        double acc = 0.0;
        for (int j = lane; j < i; j += 32) acc += xr[j] * vb[j];
        acc = warp_sum(acc);
        if (lane == 0) yb[i] = vb[i] + acc;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int k = tid; k < nb; k += blockDim.x) y[k0 + k] = yb[k];
    // rows below: four threads per row (lane bits 0–1 pick a quarter of the block's
    // columns), reduced with two shuffles
    const int q = tid & 3;
    const int64_t nrow = f - (k0 + nb);
    for (int64_t r0 = (int64_t)blockIdx.x * (blockDim.x >> 2); r0 < nrow; r0 += (int64_t)gridDim.x * (blockDim.x >> 2)) {
        const int64_t r = r0 + (tid >> 2);
        const int i = k0 + nb + (int)r;
        double acc0 = 0.0, acc1 = 0.0;
        if (r < nrow)
            for (int k = q; k < nb; k += 8) {
                acc0 += L[(int64_t)(k0 + k) * f + i] * yb[k];
                if (k + 4 < nb) acc1 += L[(int64_t)(k0 + k + 4) * f + i] * yb[k + 4];
            }
        double acc = acc0 + acc1;
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (r < nrow && q == 0) v[i] -= acc;
    }
}

__global__ void k_big_fwd_finish(int s, FactorView a, const double* __restrict__ v, const double* __restrict__ y,
                                 double* __restrict__ w) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    double* u = a.upd + a.upd_off[s];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < f; i += gridDim.x * blockDim.x) {
        if (i < c) w[first + i] = y[i] * a.dinv[first + i];
        else u[i - c] = v[i];
    }
}

// backward: v_k = w_k − Σ_{i ≥ c} L_ik xp_{R_i} for the pivot rows (one warp per k)
__global__ void k_big_bwd_below(int s, FactorView a, const double* __restrict__ w, const double* __restrict__ xp,
                                double* __restrict__ v) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int* R = a.rows + a.row_ptr[s];
    const double* L = a.front + a.front_off[s];
    const int lane = threadIdx.x & 31;
    const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= c) return;
    const double* colk = L + (int64_t)k * f;
    double acc = 0.0;
    for (int i = c + lane; i < f; i += 32) acc += colk[i] * xp[R[i]];
    acc = warp_sum(acc);
    if (lane == 0) v[k] = w[first + k] - acc;
}

// one backward block (from the last): x_b = L_bb⁻ᵀ v_b with the stored inverse (every
// CTA, redundantly), CTA 0 stores x_b; each CTA updates its rows k < k0:
// v_k −= Σ_j L_{k0+j,k} x_j
__global__ void __launch_bounds__(256) k_big_bwd_step(int s, int k0, int nb, FactorView a,
                                                      const double* __restrict__ Xb, double* __restrict__ v,
                                                      double* __restrict__ x) {
    __shared__ double vb[kBigNB], xb[kBigNB];
    const int f = a.nrow[s];
    const double* L = a.front + a.front_off[s];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k = tid; k < nb; k += blockDim.x) vb[k] = v[k0 + k];
    __syncthreads();
    for (int j = wid; j < nb; j += blockDim.x >> 5) {
        double acc = 0.0;
        for (int i = j + 1 + lane; i < nb; i += 32) acc += Xb[i * kBigNB + j] * vb[i];
        acc = warp_sum(acc);
        if (lane == 0) xb[j] = vb[j] + acc;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int k = tid; k < nb; k += blockDim.x) x[k0 + k] = xb[k];
    // earlier rows: eight threads per row k read consecutive entries of its column
    const int q = tid & 7;
    for (int r0 = blockIdx.x * (blockDim.x >> 3); r0 < k0; r0 += gridDim.x * (blockDim.x >> 3)) {
        const int k = r0 + (tid >> 3);
        double acc = 0.0;
        if (k < k0) {
            const double* colk = L + (int64_t)k * f + k0;
            for (int j = q; j < nb; j += 8) acc += colk[j] * xb[j];
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (k < k0 && q == 0) v[k] -= acc;
    }
}

__global__ void k_big_bwd_finish(int s, FactorView a, const double* __restrict__ xs, double* __restrict__ xp,
                                 double* __restrict__ x, int accumulate) {
    const int c = a.ncol[s], first = a.first[s];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
        const double xi = xs[i];
        xp[first + i] = xi;
        if (accumulate) x[a.perm[first + i]] += xi;
        else x[a.perm[first + i]] = xi;
    }
}

int g_nsm = 0;
int nsm() {
    if (!g_nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
        if (g_nsm <= 0) g_nsm = 1;
    }
    return g_nsm;
}

unsigned gridfor(int64_t n, int threads) {
    const int64_t b = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)nsm() * 16));
}

template <class T>
int big_factor_t(const FactorPlan& P, const FactorView& a, const double* kval, int idx, T* F, T* W,
                 cudaStream_t st) {
    const int s = P.big_s[idx], f = P.big_f[idx], c = P.big_c[idx];
    int launches = 0;
    const int64_t ff = (int64_t)f * f;
    k_big_zero<T><<<gridfor(ff, 256), 256, 0, st>>>(F, ff);
    k_big_assemble<T><<<gridfor(P.big_amap_n[idx], 256), 256, 0, st>>>(s, a, kval, F);
    k_big_extend_add<T><<<(unsigned)((f + 7) / 8), 256, 0, st>>>(s, a, P.d_ea_ptr + P.big_ea_off[idx],
                                                                  P.d_ea_child, P.d_ea_pos, F);
    launches += 3;
    for (int k0 = 0; k0 < c; k0 += kBigNB) {
        const int nb = std::min(kBigNB, c - k0);
        k_big_diag<T><<<1, 256, 0, st>>>(s, k0, nb, a, F, P.big_linv + P.big_linv_off[idx] +
                                                              (int64_t)(k0 / kBigNB) * kBigNB * kBigNB);
        const int rows = f - k0 - nb;
        ++launches;
        if (rows <= 0) continue;
        k_big_l21<T><<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(s, k0, nb, a, F, W);
        const int nt = (rows + kBT - 1) / kBT;
        k_big_trailing<T><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, st>>>(s, k0, nb, a, F, W);
        launches += 2;
    }
    return launches;
}

}  // namespace

int launch_big_factor(const FactorPlan& P, const FactorView& a, const double* kval, int idx, cudaStream_t st) {
    const int f = P.big_f[idx];
    const int64_t off = P.big_front_off[idx];
    int launches = 0;
    if (P.big_fp32) {
        float* F = P.big_work32;
        launches += big_factor_t<float>(P, a, kval, idx, F, (float*)P.big_w, st);
        const int64_t ff = (int64_t)f * f;
        k_big_writeback<<<gridfor(ff, 256), 256, 0, st>>>(F, a.front + off, f);
        ++launches;
    } else {
        launches += big_factor_t<double>(P, a, kval, idx, a.front + off, (double*)P.big_w, st);
    }
    return launches;
}

int launch_big_fwd(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, int idx,
                   cudaStream_t st) {
    const int s = P.big_s[idx], f = P.big_f[idx], c = P.big_c[idx];
    int launches = 0;
    k_big_fwd_gather<<<gridfor(f, 256), 256, 0, st>>>(s, a, P.d_ea_ptr + P.big_ea_off[idx], P.d_ea_child,
                                                       P.d_ea_pos, rhs, P.big_v);
    ++launches;
    for (int k0 = 0; k0 < c; k0 += kBigNB) {
        const int nb = std::min(kBigNB, c - k0);
        const double* Xb = P.big_linv + P.big_linv_off[idx] + (int64_t)(k0 / kBigNB) * kBigNB * kBigNB;
        k_big_fwd_step<<<gridfor(4 * (int64_t)std::max(1, f - k0 - nb), 256), 256, 0, st>>>(s, k0, nb, a, Xb,
                                                                                          P.big_v, P.big_y);
        ++launches;
    }
    k_big_fwd_finish<<<gridfor(f, 256), 256, 0, st>>>(s, a, P.big_v, P.big_y, w);
    return launches + 1;
}

int launch_big_bwd(const FactorPlan& P, const FactorView& a, const double* w, double* xp, double* x,
                   bool accumulate, int idx, cudaStream_t st) {
    const int s = P.big_s[idx], c = P.big_c[idx];
    int launches = 0;
    k_big_bwd_below<<<(unsigned)((c + 7) / 8), 256, 0, st>>>(s, a, w, xp, P.big_v);
    ++launches;
    const int nblk = (c + kBigNB - 1) / kBigNB;
    for (int b = nblk - 1; b >= 0; --b) {
        const int k0 = b * kBigNB, nb = std::min(kBigNB, c - k0);
        const double* Xb = P.big_linv + P.big_linv_off[idx] + (int64_t)b * kBigNB * kBigNB;
        k_big_bwd_step<<<gridfor(8 * (int64_t)std::max(1, k0), 256), 256, 0, st>>>(s, k0, nb, a, Xb, P.big_v,
                                                                                 P.big_y);
        ++launches;
    }
    k_big_bwd_finish<<<gridfor(c, 256), 256, 0, st>>>(s, a, P.big_y, xp, x, accumulate ? 1 : 0);
    return launches + 1;
}

}  // namespace qoco
