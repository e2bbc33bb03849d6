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
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "common.cuh"
#include "factor.h"

namespace qoco {

namespace {

int nsm();               // SM count of the current device (queried once, outside captures)

// largest magnitude a scaled FP32 front's L, D or update entry may reach before the
// factor counts as broken down: near the FP32 overflow threshold (entries well above the
// FP64 factor's, up to 1e20 and more, still make a usable preconditioner when pivots
// were floored)
constexpr double kFp32Growth = 1e30;

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
        const int64_t off = a.amap_off[e];
        double v = kval[a.amap_slot[e]];
        const int col = (int)(off / f), row = (int)(off - (int64_t)col * f);
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
__global__ void __launch_bounds__(256) k_big_diag(int s, int k0, int nb, FactorView a, T* __restrict__ F) {
    constexpr int kOwn = (kBigNB * (kBigNB + 1) / 2 + 255) / 256;  // entries per thread
    __shared__ T D[kBigNB][kBigNB + 1];
    __shared__ T s_inv[kBigNB];
    __shared__ signed char s_sign[kBigNB];
    const int f = a.nrow[s], first = a.first[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ntri = nb * (nb + 1) / 2;
    // pivot signs staged once, off the pivot chain
    for (int k = tid; k < nb; k += nt) s_sign[k] = a.dsign[first + k0 + k] > 0 ? 1 : -1;
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
    // FP32 fronts are scaled so that no entry exceeds 1: a pivot below the floor *piv32
    // there is rounding noise of the FP32 elimination, and is replaced like a breakdown
    const double floor32 = sizeof(T) == 4 ? *a.piv32 : 0.0;
    const T thr = (T)fmax(a.dyn_thresh, floor32);
    const T dval = (T)fmax(a.dyn_value, floor32);
    auto pivot = [&](int k) {
        T d = D[k][k];
        const bool pos = s_sign[k] > 0;
        const bool ok = pos ? (d >= thr) : (d <= -thr);
        if (!ok) { d = pos ? dval : -dval; ++nreg; }
        D[k][k] = d;
        s_inv[k] = rcp_t<T>(d);
    };
    // which diagonal entries this thread owns (entry (d, d) has index d(d+3)/2)
    uint64_t own_diag = 0;
#pragma unroll
    for (int u = 0; u < kOwn; ++u)
        if (oi[u] >= 0 && oi[u] == oj[u]) own_diag |= 1ull << oi[u];
    if (own_diag & 1ull) pivot(0);
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        const T inv = s_inv[k];
        // the next pivot first: its owner updates it and computes it before anything else
        if (k + 1 < nb && ((own_diag >> (k + 1)) & 1ull)) {
            D[k + 1][k + 1] -= D[k + 1][k] * D[k + 1][k] * inv;
            pivot(k + 1);
        }
#pragma unroll
        for (int u = 0; u < kOwn; ++u) {
            const int i = oi[u], j = oj[u];
            if (j <= k || (i == k + 1 && j == k + 1)) continue;
            D[i][j] -= D[i][k] * D[j][k] * inv;
        }
        __syncthreads();
    }
    // FP64 reciprocal pivots for the solves (off the pivot chain)
    for (int k = tid; k < nb; k += nt) a.dinv[first + k0 + k] = recip((double)D[k][k]);
    // L (scaled columns) and D back to the front
    for (int t = tid; t < nb * nb; t += nt) {
        const int j = t / nb, i = t - j * nb;
        if (i > j) F[(int64_t)(k0 + j) * f + k0 + i] = D[i][j] * s_inv[j];
        else if (i == j) F[(int64_t)(k0 + j) * f + k0 + i] = D[i][j];
    }
    if (nreg) atomicAdd(a.nreg, nreg);
}

// X = L11⁻¹ of a panel's unit-lower diagonal block, row-major X[i·kBigNB + j], stored
// in the solves' block-inverse slot; one warp per column j of X (x = e_j, then for
// k = j … nb−1 the rows i > k take x_i −= L_ik·x_k).  The panel's rows below use it
// right away (k_big_l21x): their triangular solves become one parallel product.
template <class T>
__device__ __forceinline__ void panel_inverse_body(int s, int k0, int nb, const FactorView& a, const T* __restrict__ F,
                                                   double* __restrict__ X, int jblock) {
    __shared__ double L[kBigNB][kBigNB + 1];
    __shared__ double xs[8][kBigNB];
    const int f = a.nrow[s];
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int j = t / nb, i = t - j * nb;
        L[i][j] = i > j ? (double)F[(int64_t)(k0 + j) * f + k0 + i] : 0.0;
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = jblock * 8 + w;
    if (j >= kBigNB) return;
    double* x = xs[w];
    for (int i = lane; i < kBigNB; i += 32) x[i] = i == j ? 1.0 : 0.0;
    __syncwarp();
    for (int k = j; k < nb - 1; ++k) {
        const double xk = x[k];
        for (int i = k + 1 + lane; i < nb; i += 32) x[i] -= L[i][k] * xk;
        __syncwarp();
    }
    for (int i = lane; i < kBigNB; i += 32) X[(int64_t)i * kBigNB + j] = x[i];
}
template <class T>
__global__ void __launch_bounds__(256) k_big_panel_inverse(int s, int k0, int nb, FactorView a,
                                                           const T* __restrict__ F, double* __restrict__ X) {
    panel_inverse_body<T>(s, k0, nb, a, F, X, blockIdx.x);
}
// every pivot block's inverse at once (blockIdx.y = block), from the finished FP64 front
__global__ void __launch_bounds__(256) k_big_panel_inverse_all(int s, FactorView a, const double* __restrict__ F,
                                                               double* __restrict__ Xall) {
    const int c = a.ncol[s], k0 = blockIdx.y * kBigNB;
    panel_inverse_body<double>(s, k0, min(kBigNB, c - k0), a, F, Xall + (int64_t)blockIdx.y * kBigNB * kBigNB,
                               blockIdx.x);
}

// Tensor-core operands of an FP32 front's outer panel, row-major with leading dimension
// ldw: each FP32 value v split into a TF32 head (v with its 13 low mantissa bits cleared)
// and the FP32 remainder v − head (exact).  Null pointers for FP64 fronts.
struct SplitOut {
    float* Lhi = nullptr;
    float* Llo = nullptr;
    float* Whi = nullptr;
    float* Wlo = nullptr;
    int zero_to = 0;  // columns [nb, zero_to) of the split operands are written as zeros
};
__device__ __forceinline__ float tf32_head(float v) { return __uint_as_float(__float_as_uint(v) & 0xffffe000u); }

// rows i ≥ k0+nb: w_i = a_i·L11⁻ᵀ = Σ_{j ≤ k} a_ij X_kj, l_i = w_i D⁻¹ into F, w_i into
// W[i·ldw + k], and (FP32 fronts) the TF32 splits of l_i and w_i into sp at the same
// positions.  CTA: 8 rows; thread (r, g) takes row r and columns 4g … 4g+3.
template <class T>
__global__ void __launch_bounds__(128) k_big_l21x(int s, int k0, int nb, FactorView a, T* __restrict__ F,
                                                  T* __restrict__ W, SplitOut sp, int ldw,
                                                  const double* __restrict__ X) {
    __shared__ T Xs[kBigNB][kBigNB + 1];
    __shared__ T As[8][kBigNB + 1];
    __shared__ T dv[kBigNB];
    const int f = a.nrow[s], first = a.first[s];
    const int row0 = k0 + nb + blockIdx.x * 8;
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int k = t / nb, j = t - k * nb;
        Xs[k][j] = (T)X[k * kBigNB + j];
    }
    for (int t = threadIdx.x; t < 8 * nb; t += blockDim.x) {
        const int j = t >> 3, r = t & 7;
        As[r][j] = row0 + r < f ? F[(int64_t)(k0 + j) * f + row0 + r] : T(0);
    }
    for (int k = threadIdx.x; k < nb; k += blockDim.x) dv[k] = (T)a.dinv[first + k0 + k];
    __syncthreads();
    const int r = threadIdx.x & 7, g = threadIdx.x >> 3;
    const int i = row0 + r;
    if (i >= f) return;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int k = 4 * g + v;
        const int64_t o = (int64_t)i * ldw + k;
        if (k >= nb) {
            if (sp.Lhi && k < sp.zero_to) sp.Lhi[o] = sp.Llo[o] = sp.Whi[o] = sp.Wlo[o] = 0.0f;
            continue;
        }
        T acc = T(0);
        for (int j = 0; j <= k; ++j) acc += As[r][j] * Xs[k][j];
        W[o] = acc;
        const T l = acc * dv[k];
        F[(int64_t)(k0 + k) * f + i] = l;
        if (sp.Lhi) {
            const float lf = (float)l, wf = (float)acc;
            const float lh = tf32_head(lf), wh = tf32_head(wf);
            sp.Lhi[o] = lh;
            sp.Llo[o] = lf - lh;
            sp.Whi[o] = wh;
            sp.Wlo[o] = wf - wh;
        }
    }
}

// FP32 fronts: rows i ≥ k0+nb solved by forward substitution with the panel's unit-lower
// diagonal block (w_i = a_i·L11⁻ᵀ, one thread per row, the block in shared memory, w in
// registers), l_i = w_i D⁻¹ into F, w_i into W and the TF32 splits of both into sp.  No
// explicit inverse of L11: with the scaled front's pivots down to the FP32 floor, such an
// inverse can exceed the FP32 range where the substitution stays bounded.
__global__ void __launch_bounds__(128) k_big_l21_subst(int s, int k0, int nb, FactorView a, float* __restrict__ F,
                                                       float* __restrict__ W, SplitOut sp, int ldw) {
    __shared__ float Ls[kBigNB][kBigNB + 1];
    __shared__ float dv[kBigNB];
    const int f = a.nrow[s], first = a.first[s];
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int j = t / nb, i = t - j * nb;
        Ls[i][j] = i > j ? F[(int64_t)(k0 + j) * f + k0 + i] : 0.0f;
    }
    for (int k = threadIdx.x; k < kBigNB; k += blockDim.x) dv[k] = k < nb ? (float)a.dinv[first + k0 + k] : 0.0f;
    __syncthreads();
    const int i = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f) return;
    float w[kBigNB];
#pragma unroll
    for (int k = 0; k < kBigNB; ++k) w[k] = k < nb ? F[(int64_t)(k0 + k) * f + i] : 0.0f;
#pragma unroll
    for (int k = 1; k < kBigNB; ++k) {
        float acc = w[k];
#pragma unroll
        for (int j = 0; j < k; ++j) acc -= Ls[k][j] * w[j];
        w[k] = acc;
    }
    float* Wi = W + (int64_t)i * ldw;
#pragma unroll
    for (int k = 0; k < kBigNB; ++k) {
        const int64_t o = (int64_t)i * ldw + k;
        if (k < nb) {
            const float l = w[k] * dv[k];
            Wi[k] = w[k];
            F[(int64_t)(k0 + k) * f + i] = l;
            const float lh = tf32_head(l), wh = tf32_head(w[k]);
            sp.Lhi[o] = lh;
            sp.Llo[o] = l - lh;
            sp.Whi[o] = wh;
            sp.Wlo[o] = w[k] - wh;
        } else if (k < sp.zero_to) {
            sp.Lhi[o] = sp.Llo[o] = sp.Whi[o] = sp.Wlo[o] = 0.0f;
        }
    }
}

// A22 −= L21·Wᵀ on the lower triangle of rows/columns [base, f); one CTA per BT×BT tile
// of the lower triangle (tile index → (ti, tj), ti ≥ tj), (BT/R)² threads, R×R entries
// each.  Large fronts take 64-row tiles; small trailing matrices take smaller tiles so
// that the update spreads over more SMs (an SM's FP64 rate bounds a tile's time).
template <class T, int BT, int R>
__global__ void __launch_bounds__((BT / R) * (BT / R)) k_big_trailing(int s, int k0, int nb, FactorView a,
                                                                      T* __restrict__ F, const T* __restrict__ W,
                                                                      int ldw, int cend) {
    constexpr int KC = 32;  // panel columns staged per step (keeps the tiles ≤ 33 KB)
    constexpr int TX = BT / R, NTH = TX * TX;
    __shared__ T Ls[KC][BT + 1];
    __shared__ T Ws[KC][BT + 1];
    const int f = a.nrow[s];
    const int base = k0 + nb;
    const int t = blockIdx.x;
    int ti, tj;
    if (cend >= f) {
        // the whole trailing lower triangle: triangular tile index
        ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while (ti * (ti + 1) / 2 > t) --ti;
        tj = t - ti * (ti + 1) / 2;
    } else {
        // only columns [base, cend): rectangular tile grid, tiles above the diagonal idle
        const int ntj = (cend - base + BT - 1) / BT;
        ti = t / ntj;
        tj = t - ti * ntj;
        if (ti < tj) return;
    }
    const int r0 = base + ti * BT, c0 = base + tj * BT;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    T acc[R][R];
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < R; ++v) acc[u][v] = T(0);
    for (int kc = 0; kc < nb; kc += KC) {
        const int kn = min(KC, nb - kc);
        for (int e = tid; e < kn * BT; e += NTH) {
            const int k = e / BT, r = e - k * BT;
            Ls[k][r] = r0 + r < f ? F[(int64_t)(k0 + kc + k) * f + r0 + r] : T(0);
        }
        for (int e = tid; e < kn * BT; e += NTH) {
            const int cc = e / kn, k = e - cc * kn;
            Ws[k][cc] = c0 + cc < f ? W[(int64_t)(c0 + cc) * ldw + kc + k] : T(0);
        }
        __syncthreads();
        for (int k = 0; k < kn; ++k) {
            T lr[R], wc[R];
#pragma unroll
            for (int u = 0; u < R; ++u) lr[u] = Ls[k][tx + TX * u];
#pragma unroll
            for (int v = 0; v < R; ++v) wc[v] = Ws[k][ty * R + v];
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int v = 0; v < R; ++v) acc[u][v] += lr[u] * wc[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < R; ++v) {
        const int j = c0 + ty * R + v;
        if (j >= f || j >= cend) continue;
        T* Fj = F + (int64_t)j * f;
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = r0 + tx + TX * u;
            if (i < f && i >= j) Fj[i] -= acc[u][v];
        }
    }
}

// Trailing update after the panel (k0, nb) on rows [k0+nb, f) and columns [k0+nb, cend):
// the largest tile that still gives at least two CTAs per SM
template <class T>
int launch_trailing(int s, int k0, int nb, int rows, int cend, const FactorView& a, T* F, const T* W, int ldw,
                    int f, cudaStream_t st) {
    const int base = k0 + nb;
    auto ntiles = [&](int bt) -> int64_t {
        const int64_t nr = (rows + bt - 1) / bt;
        if (cend >= f) return nr * (nr + 1) / 2;
        return nr * ((cend - base + bt - 1) / bt);
    };
    const int64_t want = 2 * (int64_t)nsm();
    if (ntiles(64) >= want)
        k_big_trailing<T, 64, 4><<<(unsigned)ntiles(64), 256, 0, st>>>(s, k0, nb, a, F, W, ldw, cend);
    else if (ntiles(32) >= want)
        k_big_trailing<T, 32, 2><<<(unsigned)ntiles(32), 256, 0, st>>>(s, k0, nb, a, F, W, ldw, cend);
    else
        k_big_trailing<T, 16, 2><<<(unsigned)ntiles(16), 64, 0, st>>>(s, k0, nb, a, F, W, ldw, cend);
    return 1;
}

// ---- tensor-core trailing update (FP32 fronts) ---------------------------------------
// A22 −= L21·Wᵀ on the lower triangle of the trailing matrix after an outer panel of K ≤ 256
// columns, with tcgen05.mma kind::tf32: each FP32 operand is split into a TF32 head and its
// FP32 remainder (written by k_big_l21x), and D = Lhi·Whiᵀ + Lhi·Wloᵀ + Llo·Whiᵀ accumulates
// in FP32 in tensor memory, which keeps the update at FP32 accuracy (three TF32 products,
// the split of Ootomo & Yokota 2022).
//
// Persistent and warp-specialised, one CTA per SM (192 KB of shared memory):
//   warp 0   one thread issues the TMA loads (cp.async.bulk.tensor, 128-byte swizzle) of
//            each 32-column K chunk of the tile's four operands (Lhi, Llo: 128 rows; Whi,
//            Wlo: 256 rows) into a two-stage ring, signalling "full" through an mbarrier's
//            transaction count;
//   warp 1   owns the tensor memory (512 columns: two 128×256 FP32 accumulators) and one
//            thread issues the 12 MMAs of each chunk (4 K-steps of 8 × 3 products), then
//            commits to the stage's "empty" barrier and, after a tile's last chunk, to the
//            accumulator's "full" barrier;
//   warps 2–5 the epilogue: each warp reads its 32 tensor-memory lanes (tcgen05.ld, 32
//            columns at a time) and subtracts them from the front (column-major, coalesced
//            per column), then releases the accumulator; with two accumulators the
//            epilogue of one tile overlaps the MMAs of the next.
// Tiles are 128 rows × 256 columns of the lower triangle, in groups of 16 row blocks,
// column blocks outer within a group (the ~152 tiles in flight share their operands in L2).
// Every mbarrier wait is bounded: a wait that runs out raises *err (the solve then returns
// DEVICE_TIMEOUT) and an abort flag that ends the other roles' waits; before the CTA exits,
// its armed TMA copies and issued MMAs are waited for (bounded) and the tensor memory freed.
constexpr int kTcBM = 128, kTcBN = 256, kTcBK = 32;        // tile rows, columns; K floats per chunk
constexpr int kTcABytes = kTcBM * kTcBK * 4;               // 16 KB: one 128-row operand chunk
constexpr int kTcBBytes = kTcBN * kTcBK * 4;               // 32 KB: one 256-row operand chunk
constexpr int kTcStageBytes = 2 * kTcABytes + 2 * kTcBBytes;
constexpr int kTcStages = 2;
constexpr int kTcSmem = kTcStages * kTcStageBytes + 1024;  // + alignment slack (1024-byte atoms)
constexpr int kTcGroup = 16;                               // row blocks per tile group
constexpr long long kTcMaxPolls = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand written by TMA with the 128-byte
// swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart (stride byte offset), the
// leading byte offset unused inside one swizzle atom, descriptor version 1, layout code 2.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (16 B, unused)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                 // descriptor version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait; false when it ran out (err and abort raised) or another role aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, int* err) {
    for (long long it = 0; it < kTcMaxPolls; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
    }
    *abort = 1;
    atomicExch(err, 1);
    return false;
}

// tile t of the trailing lower triangle (row blocks of 128, column blocks of 256; block
// (ti, tj) holds entries on or below the diagonal when ti ≥ 2·tj) → (ti, tj)
__device__ __forceinline__ void tc_tile(int t, int nti, int& ti, int& tj) {
    for (int g0 = 0; g0 < nti; g0 += kTcGroup) {
        const int g1 = min(nti, g0 + kTcGroup), W = g1 - g0;
        const int T0 = g0 / 2 + 1, T1 = (g1 + 1) / 2;  // tj < T0: whole group; T0 ≤ tj < T1: ti ≥ 2tj
        const int full = T0 * W;
        const int cnt = full + (T1 - T0) * (g1 - T0 - T1 + 1);
        if (t >= cnt) { t -= cnt; continue; }
        if (t < full) { tj = t / W; ti = g0 + t % W; return; }
        t -= full;
        for (int u = T0; u < T1; ++u) {
            const int c = g1 - 2 * u;
            if (t < c) { tj = u; ti = 2 * u + t; return; }
            t -= c;
        }
    }
    ti = tj = 0;  // not reached for t < tile count
}

int tc_tile_count(int nti) {
    int n = 0;
    for (int g0 = 0; g0 < nti; g0 += kTcGroup) {
        const int g1 = std::min(nti, g0 + kTcGroup), W = g1 - g0;
        const int T0 = g0 / 2 + 1, T1 = (g1 + 1) / 2;
        n += T0 * W + (T1 - T0) * (g1 - T0 - T1 + 1);
    }
    return n;
}

struct TcMaps {
    CUtensorMap Lhi, Llo, Whi, Wlo;
};

__global__ void __launch_bounds__(192, 1) k_big_trailing_tma(const __grid_constant__ TcMaps maps,
                                                             float* __restrict__ F, int f, int base, int nchunk,
                                                             int nti, int ntile, int* err) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar_full[kTcStages], bar_empty[kTcStages], bar_tfull[2], bar_tempty[2],
        bar_drain;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < kTcStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_empty[i])));
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_tfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&bar_tempty[i])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar_drain)));
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.Lhi) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.Llo) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.Whi) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.Wlo) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const int m = f - base;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int g = 0;          // chunks issued so far (over all tiles)
        int armed[kTcStages] = {-1, -1};
        bool ok = true;
        for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
            int ti, tj;
            tc_tile(t, nti, ti, tj);
            const int ra = base + ti * kTcBM, rb = base + tj * kTcBN;
            for (int c = 0; c < nchunk && ok; ++c, ++g) {
                const int st = g % kTcStages;
                if (!(ok = mbar_wait(smem_u32(&bar_empty[st]), ((g / kTcStages) & 1) ^ 1, &s_abort, err))) break;
                const uint32_t fb = smem_u32(&bar_full[st]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kTcStageBytes)
                             : "memory");
                armed[st] = g;
                unsigned char* sb = sm + st * kTcStageBytes;
                const int x = c * kTcBK;
                const CUtensorMap* tm[4] = {&maps.Lhi, &maps.Llo, &maps.Whi, &maps.Wlo};
                const uint32_t dst[4] = {smem_u32(sb), smem_u32(sb + kTcABytes), smem_u32(sb + 2 * kTcABytes),
                                         smem_u32(sb + 2 * kTcABytes + kTcBBytes)};
                const int y[4] = {ra, ra, rb, rb};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                        ::"r"(dst[q]), "l"((uint64_t)tm[q]), "r"(x), "r"(y[q]), "r"(fb)
                        : "memory");
            }
        }
        if (!ok) {
            // copies already armed must land before the CTA leaves
            for (int st = 0; st < kTcStages; ++st)
                if (armed[st] >= 0) {
                    const uint32_t fb = smem_u32(&bar_full[st]);
                    const uint32_t par = (armed[st] / kTcStages) & 1;
                    for (long long it = 0; it < kTcMaxPolls && !mbar_try(fb, par); ++it) {}
                }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        // D format F32, A and B TF32, both K-major, N = 256, M = 128
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcBN >> 3) << 17) |
                               ((uint32_t)(kTcBM >> 4) << 24);
        int g = 0, n = 0;
        bool ok = true, issued = false;
        for (int t = blockIdx.x; t < ntile && ok; t += gridDim.x, ++n) {
            const int b = n & 1;
            if (!(ok = mbar_wait(smem_u32(&bar_tempty[b]), ((n >> 1) & 1) ^ 1, &s_abort, err))) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d = tmem + (uint32_t)(b * kTcBN);
            for (int c = 0; c < nchunk; ++c, ++g) {
                const int st = g % kTcStages;
                if (!(ok = mbar_wait(smem_u32(&bar_full[st]), (g / kTcStages) & 1, &s_abort, err))) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sb = smem_u32(sm + st * kTcStageBytes);
                const uint32_t Ahi = sb, Alo = sb + kTcABytes, Bhi = sb + 2 * kTcABytes,
                               Blo = sb + 2 * kTcABytes + kTcBBytes;
                const uint32_t As[3] = {Ahi, Ahi, Alo}, Bs[3] = {Bhi, Blo, Bhi};
#pragma unroll
                for (int ks = 0; ks < kTcBK / 8; ++ks)
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const uint64_t ad = umma_desc_sw128(As[q] + ks * 32);
                        const uint64_t bd = umma_desc_sw128(Bs[q] + ks * 32);
                        const uint32_t acc = (c > 0 || ks > 0 || q > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                    }
                issued = true;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&bar_empty[st]))
                             : "memory");
            }
            if (!ok) break;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar_tfull[b]))
                         : "memory");
        }
        if (!ok && issued) {
            // MMAs already issued must finish before the tensor memory is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar_drain))
                         : "memory");
            for (long long it = 0; it < kTcMaxPolls && !mbar_try(smem_u32(&bar_drain), 0); ++it) {}
        }
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads tensor-memory lanes 32·(w mod 4) …
        const int quarter = warp & 3;
        int n = 0;
        for (int t = blockIdx.x; t < ntile; t += gridDim.x, ++n) {
            const int b = n & 1;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(smem_u32(&bar_tfull[b]), (n >> 1) & 1, &s_abort, err);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            int ti, tj;
            tc_tile(t, nti, ti, tj);
            const int r0 = ti * kTcBM, c0 = tj * kTcBN;  // relative to base
            const int i = r0 + quarter * 32 + lane;
            const bool row_ok = i < m;
            float* Fi = F + (int64_t)base * f + base + i;  // column `base` of row base + i
            for (int cb = 0; cb < kTcBN / 32; ++cb) {
                const int j0 = c0 + cb * 32;
                if (j0 > r0 + kTcBM - 1 || j0 >= m) break;  // chunk wholly above the diagonal / past the end
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kTcBN + cb * 32);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                      "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float old[32];
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = j0 + jj;
                    old[jj] = (row_ok && j < m && i >= j) ? Fi[(int64_t)j * f] : 0.0f;
                }
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = j0 + jj;
                    if (row_ok && j < m && i >= j) Fi[(int64_t)j * f] = old[jj] - __uint_as_float(v[jj]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_tempty[b])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// ---- leaf groups ----------------------------------------------------------------------
// Member pivots: one warp per member front (childless, c ≤ 8 pivot columns): its f×c
// columns are assembled from the KKT values, the c×c block factored (dynamic
// regularisation as everywhere), the columns scaled to L; the update block is never
// formed (its sum over the group reaches the parent through k_group_syrk_*).
__global__ void k_leaf_members(const int* __restrict__ members, int nmem, FactorView a,
                               const double* __restrict__ kval) {
    const int lane = threadIdx.x & 31;
    const int w = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= nmem) return;
    const int s = members[w];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    double* Fm = a.front + a.front_off[s];
    for (int e = lane; e < f * c; e += 32) Fm[e] = 0.0;
    __syncwarp();
    for (int64_t e = a.amap_ptr[s] + lane; e < a.amap_ptr[s + 1]; e += 32) {
        const int off = (int)a.amap_off[e];  // a member front: f·c < 2^31
        double v = kval[a.amap_slot[e]];
        const int col = off / f, row = off - col * f;
        if (row == col) v += a.dsign[first + col] > 0 ? a.eps : -a.eps;
        Fm[off] = v;
    }
    __syncwarp();
    int nreg = 0;
    for (int k = 0; k < c; ++k) {
        double d = Fm[k * f + k];
        const bool pos = a.dsign[first + k] > 0;
        const bool ok = pos ? (d >= a.dyn_thresh) : (d <= -a.dyn_thresh);
        if (!ok) { d = pos ? a.dyn_value : -a.dyn_value; ++nreg; }
        const double inv = recip(d);
        __syncwarp();
        if (lane == 0) {
            Fm[k * f + k] = d;
            a.dinv[first + k] = inv;
        }
        // later pivot columns with the unscaled column k, then scale column k
        for (int j = k + 1; j < c; ++j) {
            const double wj = Fm[k * f + j] * inv;
            for (int i = j + lane; i < f; i += 32) Fm[j * f + i] -= Fm[k * f + i] * wj;
        }
        __syncwarp();
        for (int i = k + 1 + lane; i < f; i += 32) Fm[k * f + i] *= inv;
        __syncwarp();
    }
    if (lane == 0 && nreg) atomicAdd(a.nreg, nreg);
}

// Group operands, one warp per gathered column k (member column p of member m):
// Lg[k·r + i] = L21(i, p), Wg[k·r + i] = L21(i, p)·d_p
__global__ void k_group_gather(const int* __restrict__ members, const int* __restrict__ gmem,
                               const int* __restrict__ gloc, int K, int r, FactorView a, double* __restrict__ Lg,
                               double* __restrict__ Wg) {
    const int lane = threadIdx.x & 31;
    const int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (k >= K) return;
    const int s = members[gmem[k]], p = gloc[k];
    const int f = a.nrow[s], c = a.ncol[s];
    const double* col = a.front + a.front_off[s] + (int64_t)p * f;
    const double d = col[p];
    for (int i = lane; i < r; i += 32) {
        const double l = col[c + i];
        Lg[(int64_t)k * r + i] = l;
        Wg[(int64_t)k * r + i] = l * d;
    }
}

// Split-K partial products of the group's update −Lg·Wgᵀ (a contraction over the K
// gathered columns, FP64 FMA-bound): CTA (tile, split) computes one kGT×kGT lower tile
// of Lgᵀ·Wg over its K-chunk into part[(split·ntile + tile)·kGT²].  Small tiles keep the
// work spent on the upper halves of diagonal tiles and on the ragged last tile row low.
constexpr int kGT = kGroupTile;
__device__ __forceinline__ void lower_tile(int tile, int& ti, int& tj) {
    ti = (int)((sqrtf(8.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
    while (ti * (ti + 1) / 2 > tile) --ti;
    tj = tile - ti * (ti + 1) / 2;
}
__global__ void __launch_bounds__(64) k_group_syrk_part(const double* __restrict__ Lg, const double* __restrict__ Wg,
                                                        int r, int K, int nsplit, double* __restrict__ part) {
    constexpr int KC = 32;
    __shared__ double Ls[KC][kGT + 1];
    __shared__ double Ws[KC][kGT + 1];
    const int nt = (r + kGT - 1) / kGT, ntile = nt * (nt + 1) / 2;
    const int tile = blockIdx.x % ntile, split = blockIdx.x / ntile;
    int ti, tj;
    lower_tile(tile, ti, tj);
    const int r0 = ti * kGT, c0 = tj * kGT;
    const int kchunk = (K + nsplit - 1) / nsplit;
    const int kb = split * kchunk, ke = min(K, kb + kchunk);
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;  // rows tx, tx+8; columns 2ty, 2ty+1
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int k0 = kb; k0 < ke; k0 += KC) {
        const int kn = min(KC, ke - k0);
        for (int e = tid; e < KC * kGT; e += 64) {
            const int k = e / kGT, rr = e - k * kGT;
            const bool in = k < kn;
            Ls[k][rr] = (in && r0 + rr < r) ? Lg[(int64_t)(k0 + k) * r + r0 + rr] : 0.0;
            Ws[k][rr] = (in && c0 + rr < r) ? Wg[(int64_t)(k0 + k) * r + c0 + rr] : 0.0;
        }
        __syncthreads();
        for (int k = 0; k < kn; ++k) {
            const double l0 = Ls[k][tx], l1 = Ls[k][tx + 8];
            const double w0 = Ws[k][2 * ty], w1 = Ws[k][2 * ty + 1];
            acc[0][0] += l0 * w0;
            acc[0][1] += l0 * w1;
            acc[1][0] += l1 * w0;
            acc[1][1] += l1 * w1;
        }
        __syncthreads();
    }
    double* out = part + ((int64_t)split * ntile + tile) * (kGT * kGT);
    out[tx * kGT + 2 * ty] = acc[0][0];
    out[tx * kGT + 2 * ty + 1] = acc[0][1];
    out[(tx + 8) * kGT + 2 * ty] = acc[1][0];
    out[(tx + 8) * kGT + 2 * ty + 1] = acc[1][1];
}

// Sum of the split-K partials in split order, subtracted into the parent front at the
// members' relative positions (lower triangle)
template <class T>
__global__ void k_group_syrk_reduce(const double* __restrict__ part, int r, int nsplit, const int* __restrict__ rel,
                                    int f, T* __restrict__ F) {
    const int nt = (r + kGT - 1) / kGT, ntile = nt * (nt + 1) / 2;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ntile * kGT * kGT) return;
    const int tile = (int)(e / (kGT * kGT)), q = (int)(e - (int64_t)tile * kGT * kGT);
    int ti, tj;
    lower_tile(tile, ti, tj);
    const int i = ti * kGT + q / kGT, j = tj * kGT + q % kGT;
    if (i >= r || j >= r || i < j) return;
    double sum = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) sum += part[((int64_t)sp * ntile + tile) * (kGT * kGT) + q];
    F[(int64_t)rel[j] * f + rel[i]] -= (T)sum;
}

// FP32 fronts are factored scaled: with σ_i = 1/√(max_j |G_ij|) of the assembled FP64
// front G (one pass of Ruiz's symmetric equilibration in the max norm), every entry of
// F = ΣGΣ is at most 1 in magnitude (|G_ij| ≤ min(r_i, r_j) ≤ √(r_i r_j), r the row
// maxima), whatever the spread of the −W² block (1e±16 near the end of a solve), and its
// LDLᵀ (L̃, D̃) gives G's as L = Σ⁻¹L̃Σ, D = Σ⁻¹D̃Σ⁻¹, update block Σ⁻¹ŨΣ⁻¹.  (Scaling to
// a unit diagonal instead leaves off-diagonal entries up to 1e8 where the diagonal is the
// static regularisation alone, and the FP32 elimination's growth from them breaks it down.)
// One CTA per 64 rows: the rows' entries left of the diagonal are read as 64-row strips of
// the columns j ≤ i (contiguous per column), the entries below the diagonal as the rows'
// own columns; every block reads about 64·f entries and no atomics are needed.
constexpr int kScaleRows = 64;
__global__ void __launch_bounds__(256) k_big_scale(const double* __restrict__ G, int f, double* __restrict__ sc) {
    __shared__ double part[4][kScaleRows];
    __shared__ double colm[kScaleRows];
    const int i0 = blockIdx.x * kScaleRows;
    const int r = threadIdx.x % kScaleRows, p = threadIdx.x / kScaleRows;
    const int i = i0 + r;
    double m = 0.0;
    if (i < f)
        for (int j = p; j <= i; j += 4) m = fmax(m, fabs(G[(int64_t)j * f + i]));
    part[p][r] = m;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = w; q < kScaleRows; q += 8) {
        const int col = i0 + q;
        double cm = 0.0;
        if (col < f)
            for (int k = col + lane; k < f; k += 32) cm = fmax(cm, fabs(G[(int64_t)col * f + k]));
        for (int o = 16; o > 0; o >>= 1) cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
        if (lane == 0) colm[q] = cm;
    }
    __syncthreads();
    if (threadIdx.x < kScaleRows && i < f) {
        const double rm = fmax(fmax(fmax(part[0][r], part[1][r]), fmax(part[2][r], part[3][r])), colm[r]);
        sc[i] = (rm > 0.0 && isfinite(rm)) ? 1.0 / sqrt(rm) : 1.0;
    }
}
// F = ΣGΣ on the lower triangle (zeros above), plus the sign-aware shift δ on the
// diagonal (mixed_reg)
__global__ void k_big_to32(int s, FactorView a, const double* __restrict__ G, float* __restrict__ F, int f,
                           const double* __restrict__ sc) {
    const int first = a.first[s], c = a.ncol[s];
    const int64_t n = (int64_t)f * f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / f), i = (int)(e - (int64_t)j * f);
        double v = i >= j ? sc[i] * G[e] * sc[j] : 0.0;
        // the shift only on the pivot columns: the update block goes to the parent exact
        if (i == j && i < c && a.eps32 > 0.0) v += a.dsign[first + i] > 0 ? a.eps32 : -a.eps32;
        F[e] = (float)v;
    }
}
// factored FP32 working front → the FP64 front storage, unscaled (lower triangle); the
// reciprocal pivots of the solves recomputed from the unscaled D
__global__ void k_big_writeback(int s, FactorView a, const float* __restrict__ Fw, double* __restrict__ G, int f,
                                int c, const double* __restrict__ sc) {
    const int first = a.first[s];
    const int64_t n = (int64_t)f * f;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / f), i = (int)(e - (int64_t)j * f);
        if (i < j) continue;
        const double v = (double)Fw[e];
        bad |= !(fabs(v) <= kFp32Growth);  // also true for NaN
        if (j < c) {
            if (i == j) {
                const double d = v / (sc[j] * sc[j]);
                G[e] = d;
                a.dinv[first + j] = recip(d);
            } else {
                G[e] = v * sc[j] / sc[i];
            }
        } else {
            G[e] = v / (sc[i] * sc[j]);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.bad32, 1);
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

// Leaf-group members' update vectors, summed in two deterministic stages: CTA b sums
// members [b·kGrpChunk, …) row by row into part[b·r + i]; then the chunks are summed in
// order into the parent's gathered vector at the members' relative rows.
constexpr int kGrpChunk = 256;
__global__ void k_group_upd_part(const int64_t* __restrict__ updoff, int nmem, int r, FactorView a,
                                 double* __restrict__ part) {
    const int b = blockIdx.x;
    const int m0 = b * kGrpChunk, m1 = min(nmem, m0 + kGrpChunk);
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
        double acc = 0.0;
        for (int m = m0; m < m1; ++m) acc += a.upd[updoff[m] + i];
        part[(int64_t)b * r + i] = acc;
    }
}
__global__ void k_group_upd_reduce(const double* __restrict__ part, int nchunk, int r, const int* __restrict__ rel,
                                   double* __restrict__ v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= r) return;
    double acc = 0.0;
    for (int b = 0; b < nchunk; ++b) acc += part[(int64_t)b * r + i];
    v[rel[i]] += acc;
}

// ---- dataflow solves of one large front ----------------------------------------------
// Forward: row blocks are the pivot blocks [k0, k0+nb) (nb ≤ 64) followed by 64-row blocks
// of the border rows ≥ c, taken in that order from a counter (ctl[0]).  Block b subtracts
// L_{rows, k}·y_k for each pivot block k < b (k < nblk for a border block) as soon as y_k
// is published (flag ctl[1+k], bounded wait); a pivot block then computes
// y_b = X_b·(v_b − Σ) with its stored block inverse and publishes it, a border block
// leaves v − Σ (the front's update vector).  A block waits only on blocks taken before
// it, so the launch cannot deadlock whatever the number of resident CTAs.
constexpr int kDfThreads = 256;

__device__ __forceinline__ bool df_wait(const int* flag, int* err, long long max_spins) {
    const volatile int* vf = flag;
    const volatile int* ve = err;
    long long spins = 0;
    while (*vf == 0) {
        if (*ve) return false;
        if (++spins > max_spins) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

__device__ __forceinline__ int df_take(int* ctl) {
    __shared__ int s_b;
    if (threadIdx.x == 0) s_b = atomicAdd(ctl, 1);
    __syncthreads();
    const int b = s_b;
    __syncthreads();
    return b;
}

__global__ void __launch_bounds__(kDfThreads) k_big_fwd_df(int s, FactorView a, const double* __restrict__ Xall,
                                                           double* __restrict__ v, double* __restrict__ y,
                                                           int* __restrict__ ctl, int* err, long long max_spins) {
    __shared__ double part[4][kBigNB];
    __shared__ double ys[kBigNB];
    const int f = a.nrow[s], c = a.ncol[s];
    const double* L = a.front + a.front_off[s];
    const int nblk = (c + kBigNB - 1) / kBigNB, nrb = nblk + (f - c + kBigNB - 1) / kBigNB;
    const int tid = threadIdx.x, r = tid & (kBigNB - 1), q = tid >> 6;
    for (;;) {
        const int b = df_take(ctl);
        if (b >= nrb) return;
        const bool pivot = b < nblk;
        const int row0 = pivot ? b * kBigNB : c + (b - nblk) * kBigNB;
        const int nrow = pivot ? min(kBigNB, c - row0) : min(kBigNB, f - row0);
        const int i = row0 + r;
        const bool mine = r < nrow;
        // this thread's entries of the block inverse (final since the factorisation),
        // loaded before any wait: X_{r,j}, j = q + 4m ≤ r
        const double* X = Xall + (int64_t)(pivot ? b : 0) * kBigNB * kBigNB;
        double xv[kBigNB / 4];
#pragma unroll
        for (int m = 0; m < kBigNB / 4; ++m) {
            const int j = q + 4 * m;
            xv[m] = (pivot && mine && j <= r) ? X[r * kBigNB + j] : 0.0;
        }
        const double vi = mine ? v[i] : 0.0;  // final before the launch (pivot rows are read only)
        double acc = 0.0;
        const int kend = pivot ? b : nblk;
        for (int k = 0; k < kend; ++k) {
            const int k0 = k * kBigNB, nb = min(kBigNB, c - k0);
            // L's block (rows of b, columns of k) is final: its loads go out before the wait
            double l[kBigNB / 4];
#pragma unroll
            for (int m = 0; m < kBigNB / 4; ++m) {
                const int kk = q + 4 * m;
                l[m] = (mine && kk < nb) ? L[(int64_t)(k0 + kk) * f + i] : 0.0;
            }
            bool ok = true;
            if (tid == 0) {
                ok = df_wait(ctl + 1 + k, err, max_spins);
                __threadfence();
            }
            if (!__syncthreads_and(ok)) return;
            if (tid < kBigNB) ys[tid] = tid < nb ? __ldcg(y + k0 + tid) : 0.0;
            __syncthreads();
#pragma unroll
            for (int m = 0; m < kBigNB / 4; ++m) acc += l[m] * ys[q + 4 * m];
            __syncthreads();
        }
        part[q][r] = acc;
        __syncthreads();
        if (!pivot) {
            if (q == 0 && mine) v[i] = vi - ((part[0][r] + part[1][r]) + (part[2][r] + part[3][r]));
            __syncthreads();
            continue;
        }
        if (q == 0) ys[r] = mine ? vi - ((part[0][r] + part[1][r]) + (part[2][r] + part[3][r])) : 0.0;
        __syncthreads();
        // y_b = X_b u (X unit lower, row-major): row r, quarter q of its columns j ≤ r
        double t = 0.0;
#pragma unroll
        for (int m = 0; m < kBigNB / 4; ++m) t += xv[m] * ys[q + 4 * m];
        part[q][r] = t;
        __syncthreads();
        if (q == 0 && mine) y[i] = (part[0][r] + part[1][r]) + (part[2][r] + part[3][r]);
        __syncthreads();
        if (tid == 0) {
            __threadfence();  // cumulative: orders the block's stores (seen through the barrier) before the flag
            atomicExch(ctl + 1 + b, 1);
        }
    }
}

// Backward, pivot blocks from the last: block b (taken as nblk−1−counter) waits for every
// later block k > b, last first (the order in which they are published), and subtracts
// Σ_j L_{j,i}·x_j (column i of L, rows of block k) from v_i, then x_b = X_bᵀ·(v_b − Σ) and
// publishes it.  v holds w − (border contributions) from k_big_bwd_below.
__global__ void __launch_bounds__(kDfThreads) k_big_bwd_df(int s, FactorView a, const double* __restrict__ Xall,
                                                           const double* __restrict__ v, double* __restrict__ x,
                                                           int* __restrict__ ctl, int* err, long long max_spins) {
    __shared__ double part[8][kBigNB + 1];
    __shared__ double xs[kBigNB];
    __shared__ double us[kBigNB];
    __shared__ double red[4][kBigNB];
    const int f = a.nrow[s], c = a.ncol[s];
    const double* L = a.front + a.front_off[s];
    const int nblk = (c + kBigNB - 1) / kBigNB;
    const int tid = threadIdx.x, q8 = tid & 7, rr = tid >> 3;  // 32 rows × 8 per pass
    for (;;) {
        const int t = df_take(ctl);
        if (t >= nblk) return;
        const int b = nblk - 1 - t;
        const int row0 = b * kBigNB, nrow = min(kBigNB, c - row0);
        // this thread's entries of the block inverse, loaded before any wait:
        // X_{i,j} for column j = tid & 63 and rows i = j + q + 4m < nrow
        const int j = tid & (kBigNB - 1), q = tid >> 6;
        const double* X = Xall + (int64_t)b * kBigNB * kBigNB;
        double xv[kBigNB / 4];
#pragma unroll
        for (int m = 0; m < kBigNB / 4; ++m) {
            const int i = j + q + 4 * m;
            xv[m] = (j < nrow && i < nrow) ? X[i * kBigNB + j] : 0.0;
        }
        const double vj = (tid < kBigNB && tid < nrow) ? v[row0 + tid] : 0.0;  // read only here
        double acc0 = 0.0, acc1 = 0.0;  // rows rr and rr + 32
        // later blocks in the order they are published (the last first)
        for (int k = nblk - 1; k > b; --k) {
            const int k0 = k * kBigNB, nb = min(kBigNB, c - k0);
            // L's block is final: its loads go out before the wait
            double l0[kBigNB / 8], l1[kBigNB / 8];
            const double* col0 = L + (int64_t)(row0 + rr) * f + k0;
            const double* col1 = col0 + (int64_t)32 * f;
#pragma unroll
            for (int m = 0; m < kBigNB / 8; ++m) {
                const int j = q8 + 8 * m;
                l0[m] = (rr < nrow && j < nb) ? col0[j] : 0.0;
                l1[m] = (rr + 32 < nrow && j < nb) ? col1[j] : 0.0;
            }
            bool ok = true;
            if (tid == 0) {
                ok = df_wait(ctl + 1 + k, err, max_spins);
                __threadfence();
            }
            if (!__syncthreads_and(ok)) return;
            if (tid < kBigNB) xs[tid] = tid < nb ? __ldcg(x + k0 + tid) : 0.0;
            __syncthreads();
#pragma unroll
            for (int m = 0; m < kBigNB / 8; ++m) {
                acc0 += l0[m] * xs[q8 + 8 * m];
                acc1 += l1[m] * xs[q8 + 8 * m];
            }
            __syncthreads();
        }
        part[q8][rr] = acc0;
        part[q8][rr + 32] = acc1;
        __syncthreads();
        if (tid < kBigNB) {
            double sum = 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) sum += part[u][tid];
            us[tid] = tid < nrow ? vj - sum : 0.0;
        }
        __syncthreads();
        // x_j = Σ_{i ≥ j} X_ij u_i (X unit lower, row-major): column j, quarter q of the rows
        double tsum = 0.0;
#pragma unroll
        for (int m = 0; m < kBigNB / 4; ++m) {
            const int i = j + q + 4 * m;
            if (i < nrow) tsum += xv[m] * us[i];
        }
        red[q][j] = tsum;
        __syncthreads();
        if (q == 0 && j < nrow) x[row0 + j] = (red[0][j] + red[1][j]) + (red[2][j] + red[3][j]);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicExch(ctl + 1 + b, 1);
        }
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

constexpr int kOuterNB = 4 * kBigNB;  // FP32 fronts: outer panel width (tensor-core K)

// The front's entries: KKT values, the children's update blocks, leaf-group products.
template <class T>
int big_assemble_t(const FactorPlan& P, const FactorView& a, const double* kval, int idx, T* F, cudaStream_t st) {
    const int s = P.big_s[idx], f = P.big_f[idx];
    int launches = 0;
    const int64_t ff = (int64_t)f * f;
    k_big_zero<T><<<gridfor(ff, 256), 256, 0, st>>>(F, ff);
    k_big_assemble<T><<<gridfor(P.big_amap_n[idx], 256), 256, 0, st>>>(s, a, kval, F);
    k_big_extend_add<T><<<(unsigned)((f + 7) / 8), 256, 0, st>>>(s, a, P.d_ea_ptr + P.big_ea_off[idx],
                                                                  P.d_ea_child, P.d_ea_pos, F);
    launches += 3;
    for (const FactorPlan::LeafGroup& g : P.groups) {
        if (g.big_idx != idx) continue;
        if (g.K == 0) continue;
        k_group_gather<<<(unsigned)((g.K + 7) / 8), 256, 0, st>>>(g.d_members, g.d_gmem, g.d_gloc, g.K, g.r, a,
                                                                  P.grp_L, P.grp_W);
        const int nt = (g.r + kGT - 1) / kGT, ntile = nt * (nt + 1) / 2;
        k_group_syrk_part<<<(unsigned)(ntile * P.grp_split), 64, 0, st>>>(P.grp_L, P.grp_W, g.r, g.K, P.grp_split,
                                                                         P.grp_part);
        const int64_t ne = (int64_t)ntile * kGT * kGT;
        k_group_syrk_reduce<T><<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(P.grp_part, g.r, P.grp_split,
                                                                            a.rel + g.rel_off, f, F);
        launches += 3;
    }
    return launches;
}

// The partial LDLᵀ of the assembled front F (panels; see the file header).
template <class T>
int big_factor_t(const FactorPlan& P, const FactorView& a, int idx, T* F, T* W, cudaStream_t st) {
    const int s = P.big_s[idx], f = P.big_f[idx], c = P.big_c[idx];
    int launches = 0;
    double* linv = P.big_linv + P.big_linv_off[idx];
    if constexpr (sizeof(T) == 8) {
        // FP64: 64-column panels, each followed by the full trailing update
        for (int k0 = 0; k0 < c; k0 += kBigNB) {
            const int nb = std::min(kBigNB, c - k0);
            k_big_diag<T><<<1, 256, 0, st>>>(s, k0, nb, a, F);
            double* X = linv + (int64_t)(k0 / kBigNB) * kBigNB * kBigNB;
            k_big_panel_inverse<T><<<kBigNB / 8, 256, 0, st>>>(s, k0, nb, a, F, X);
            const int rows = f - k0 - nb;
            launches += 2;
            if (rows <= 0) continue;
            k_big_l21x<T><<<(unsigned)((rows + 7) / 8), 128, 0, st>>>(s, k0, nb, a, F, W, SplitOut(), kBigNB, X);
            launches += 1 + launch_trailing<T>(s, k0, nb, rows, f, a, F, W, kBigNB, f, st);
        }
    } else {
        // FP32: outer panels of kOuterNB columns made of 64-column inner panels; an inner
        // panel updates only the rest of its outer panel (CUDA cores) and writes the TF32
        // splits of its L and W rows, and the trailing matrix takes one rank-kOuterNB update
        // on the tensor cores (3×TF32, TMA-fed)
        const int64_t sps = (int64_t)P.max_big_f * kOuterNB;
        for (int k0 = 0; k0 < c; k0 += kOuterNB) {
            const int nbo = std::min(kOuterNB, c - k0);
            for (int k1 = k0; k1 < k0 + nbo; k1 += kBigNB) {
                const int nb = std::min(kBigNB, k0 + nbo - k1);
                k_big_diag<T><<<1, 256, 0, st>>>(s, k1, nb, a, F);
                const int rows = f - k1 - nb;
                launches += 1;
                if (rows <= 0) continue;
                SplitOut sp;
                sp.Lhi = P.big_split + (k1 - k0);
                sp.Llo = sp.Lhi + sps;
                sp.Whi = sp.Lhi + 2 * sps;
                sp.Wlo = sp.Lhi + 3 * sps;
                // the outer panel's last inner panel zero-fills its split columns up to 64 (the
                // tensor-core K chunks of 32 reach past a ragged panel end)
                sp.zero_to = (k1 + nb == k0 + nbo) ? kBigNB : 0;
                k_big_l21_subst<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(s, k1, nb, a, (float*)F,
                                                                                (float*)W + (k1 - k0), sp, kOuterNB);
                ++launches;
                const int cend = k0 + nbo;
                if (k1 + nb < cend)
                    launches += launch_trailing<T>(s, k1, nb, rows, cend, a, F, W + (k1 - k0), kOuterNB, f, st);
            }
            const int rows = f - k0 - nbo;
            if (rows > 0) {
                const int nti = (rows + kTcBM - 1) / kTcBM;
                const int ntile = tc_tile_count(nti);
                TcMaps maps;
                memcpy(&maps, P.big_tmaps, sizeof maps);
                k_big_trailing_tma<<<(unsigned)std::min(ntile, nsm()), 192, kTcSmem, st>>>(
                    maps, (float*)F, f, k0 + nbo, (nbo + kTcBK - 1) / kTcBK, nti, ntile, P.df_err);
                ++launches;
            }
        }
    }
    return launches;
}

}  // namespace

int launch_leaf_groups(const FactorPlan& P, const FactorView& a, const double* kval, cudaStream_t st) {
    int launches = 0;
    for (const FactorPlan::LeafGroup& g : P.groups) {
        k_leaf_members<<<(unsigned)((g.nmem + 7) / 8), 256, 0, st>>>(g.d_members, g.nmem, a, kval);
        ++launches;
    }
    return launches;
}

int big_set_attributes() {
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_big_trailing_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    nsm();  // queried here, outside any stream capture of the launch sequences
    return 0;
}

// Tensor maps of the four split operands (rows: max_big_f, columns: kOuterNB FP32, row
// stride kOuterNB·4 bytes; boxes of 32 columns × 128 or 256 rows, 128-byte swizzle, rows past
// the end read as zeros).  Encoded once: the buffers live as long as the solver.
int big_tma_setup(FactorPlan& P) {
    static_assert(sizeof(TcMaps) <= sizeof(P.big_tmaps), "tensor-map storage");
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    QOCO_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr));
    if (!fn || qr != cudaDriverEntryPointSuccess) return QOCO_GPU_ERR_CUDA;
    auto encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    TcMaps maps;
    CUtensorMap* out[4] = {&maps.Lhi, &maps.Llo, &maps.Whi, &maps.Wlo};
    const int64_t sps = (int64_t)P.max_big_f * kOuterNB;
    for (int q = 0; q < 4; ++q) {
        const cuuint64_t dims[2] = {(cuuint64_t)kOuterNB, (cuuint64_t)P.max_big_f};
        const cuuint64_t strides[1] = {(cuuint64_t)kOuterNB * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)(q < 2 ? kTcBM : kTcBN)};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = encode(out[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, P.big_split + q * sps, dims, strides,
                                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return QOCO_GPU_ERR_CUDA;
    }
    memcpy(P.big_tmaps, &maps, sizeof maps);
    return 0;
}

int launch_big_factor(const FactorPlan& P, const FactorView& a, const double* kval, int idx, cudaStream_t st) {
    const int f = P.big_f[idx];
    const int64_t off = P.big_front_off[idx];
    int launches = 0;
    if (P.big_fp32) {
        // assembled in FP64, scaled symmetrically (row maxima 1), factored in FP32, and
        // L, D, the update block and the diagonal blocks' inverses unscaled into FP64
        const int s = P.big_s[idx], c = P.big_c[idx];
        float* F = P.big_work32;
        double* G = a.front + off;
        const int64_t ff = (int64_t)f * f;
        QOCO_CUDA_TRY(cudaMemsetAsync(a.bad32, 0, sizeof(int), st));
        launches += big_assemble_t<double>(P, a, kval, idx, G, st);
        k_big_scale<<<(unsigned)((f + kScaleRows - 1) / kScaleRows), 256, 0, st>>>(G, f, P.big_scale);
        k_big_to32<<<gridfor(ff, 256), 256, 0, st>>>(s, a, G, F, f, P.big_scale);
        launches += 2;
        launches += big_factor_t<float>(P, a, idx, F, (float*)P.big_w, st);
        k_big_writeback<<<gridfor(ff, 256), 256, 0, st>>>(s, a, F, G, f, c, P.big_scale);
        // the solves' pivot-block inverses, from the unscaled FP64 L
        const int nblk = (c + kBigNB - 1) / kBigNB;
        if (nblk)
            k_big_panel_inverse_all<<<dim3(kBigNB / 8, nblk), 256, 0, st>>>(s, a, G, P.big_linv + P.big_linv_off[idx]);
        launches += 2;
    } else {
        launches += big_assemble_t<double>(P, a, kval, idx, a.front + off, st);
        launches += big_factor_t<double>(P, a, idx, a.front + off, (double*)P.big_w, st);
    }
    return launches;
}

int launch_big_fwd(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, int idx,
                   cudaStream_t st) {
    const int s = P.big_s[idx], f = P.big_f[idx], c = P.big_c[idx];
    int launches = 0;
    k_big_fwd_gather<<<gridfor(f, 256), 256, 0, st>>>(s, a, P.d_ea_ptr + P.big_ea_off[idx], P.d_ea_child,
                                                       P.d_ea_pos, rhs, P.big_v);
    for (const FactorPlan::LeafGroup& g : P.groups) {
        if (g.big_idx != idx) continue;
        const int nchunk = (g.nmem + kGrpChunk - 1) / kGrpChunk;
        k_group_upd_part<<<(unsigned)nchunk, 256, 0, st>>>(g.d_updoff, g.nmem, g.r, a, P.grp_part);
        k_group_upd_reduce<<<(unsigned)((g.r + 255) / 256), 256, 0, st>>>(P.grp_part, nchunk, g.r, a.rel + g.rel_off,
                                                                          P.big_v);
        launches += 2;
    }
    ++launches;
    const int nblk = (c + kBigNB - 1) / kBigNB, nrb = nblk + (f - c + kBigNB - 1) / kBigNB;
    QOCO_CUDA_TRY(cudaMemsetAsync(P.big_ctl, 0, sizeof(int) * (1 + nblk), st));
    k_big_fwd_df<<<(unsigned)std::min(nrb, 2 * nsm()), kDfThreads, 0, st>>>(
        s, a, P.big_linv + P.big_linv_off[idx], P.big_v, P.big_y, P.big_ctl, P.df_err, P.df_spins);
    k_big_fwd_finish<<<gridfor(f, 256), 256, 0, st>>>(s, a, P.big_v, P.big_y, w);
    return launches + 2;
}

int launch_big_bwd(const FactorPlan& P, const FactorView& a, const double* w, double* xp, double* x,
                   bool accumulate, int idx, cudaStream_t st) {
    const int s = P.big_s[idx], c = P.big_c[idx];
    int launches = 0;
    k_big_bwd_below<<<(unsigned)((c + 7) / 8), 256, 0, st>>>(s, a, w, xp, P.big_v);
    ++launches;
    const int nblk = (c + kBigNB - 1) / kBigNB;
    QOCO_CUDA_TRY(cudaMemsetAsync(P.big_ctl, 0, sizeof(int) * (1 + nblk), st));
    k_big_bwd_df<<<(unsigned)std::min(nblk, 2 * nsm()), kDfThreads, 0, st>>>(
        s, a, P.big_linv + P.big_linv_off[idx], P.big_v, P.big_y, P.big_ctl, P.df_err, P.df_spins);
    k_big_bwd_finish<<<gridfor(c, 256), 256, 0, st>>>(s, a, P.big_y, xp, x, accumulate ? 1 : 0);
    return launches + 2;
}

}  // namespace qoco
