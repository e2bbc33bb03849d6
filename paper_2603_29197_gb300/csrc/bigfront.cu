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
#include <cstdint>

#include "common.cuh"
#include "factor.h"

namespace qoco {

namespace {

int nsm();               // SM count of the current device (queried once, outside captures)

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
    const T thr = (T)a.dyn_thresh, dval = (T)a.dyn_value;
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
__global__ void __launch_bounds__(256) k_big_panel_inverse(int s, int k0, int nb, FactorView a,
                                                           const T* __restrict__ F, double* __restrict__ X) {
    __shared__ double L[kBigNB][kBigNB + 1];
    __shared__ double xs[8][kBigNB];
    const int f = a.nrow[s];
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int j = t / nb, i = t - j * nb;
        L[i][j] = i > j ? (double)F[(int64_t)(k0 + j) * f + k0 + i] : 0.0;
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * 8 + w;
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

// rows i ≥ k0+nb: w_i = a_i·L11⁻ᵀ = Σ_{j ≤ k} a_ij X_kj, l_i = w_i D⁻¹ into F (and, if Lr,
// row-major into Lr[i·ldw + k]), w_i into W[i·ldw + k].  CTA: 8 rows; thread (r, g) takes
// row r and columns 4g … 4g+3.
template <class T>
__global__ void __launch_bounds__(128) k_big_l21x(int s, int k0, int nb, FactorView a, T* __restrict__ F,
                                                  T* __restrict__ W, T* __restrict__ Lr, int ldw,
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
        if (k >= nb) break;
        T acc = T(0);
        for (int j = 0; j <= k; ++j) acc += As[r][j] * Xs[k][j];
        W[(int64_t)i * ldw + k] = acc;
        const T l = acc * dv[k];
        F[(int64_t)(k0 + k) * f + i] = l;
        if (Lr) Lr[(int64_t)i * ldw + k] = l;
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
// A22 −= L21·Wᵀ on 128×128 tiles of the lower triangle with tcgen05.mma kind::tf32: each
// FP32 operand is split into a TF32 head and the FP32 remainder (a = a_hi + a_lo), and
// D = A_hi·B_hiᵀ + A_hi·B_loᵀ + A_lo·B_hiᵀ accumulates in FP32 in tensor memory, which
// keeps the update at FP32 accuracy (three TF32 products).  Operands are staged by the
// CTA's threads into shared memory in the canonical K-major layout without swizzle:
// core matrices of 8 rows × 16 bytes, adjacent along K 128 bytes apart (leading byte
// offset) and along M/N 2048 bytes apart (stride byte offset).  One thread issues the
// MMAs; completion is signalled through an mbarrier whose wait is bounded (on a timeout
// the tile is left unchanged and *err is set, so the refinement rejects the factor).
constexpr int kTcM = 128;                        // tile rows (L21) and columns (W)
constexpr int kTcTile = kTcM * kBigNB * 4;      // bytes of one 128×64 FP32 operand
constexpr int kTcSmem = 4 * kTcTile + 1024;     // four operands + alignment slack

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;                   // leading byte offset (K)
    d |= (uint64_t)((8 * kBigNB * 4) >> 4) << 32;      // stride byte offset (8-row groups)
    d |= (uint64_t)1 << 46;                            // descriptor version
    return d;                                          // layout: no swizzle
}

__global__ void __launch_bounds__(512) k_big_trailing_tc(int s, int k0, int kb, FactorView a, float* __restrict__ F,
                                                         const float* __restrict__ Lr, const float* __restrict__ W,
                                                         int ldw, int* err) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* Ahi = sm;
    unsigned char* Alo = sm + kTcTile;
    unsigned char* Bhi = sm + 2 * kTcTile;
    unsigned char* Blo = sm + 3 * kTcTile;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int f = a.nrow[s];
    const int base = k0 + kb;
    const int t = blockIdx.x;
    int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int r0 = base + ti * kTcM, c0 = base + tj * kTcM;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTcM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // D format F32, A and B TF32, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcM >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    uint32_t tmem = 0;
    bool ok = true;
    // the panel's K = kb columns in chunks of kBigNB: stage, multiply, wait, next chunk
    for (int kc = 0, round = 0; kc < kb; kc += kBigNB, ++round) {
        const int kn = min(kBigNB, kb - kc);
        // operands, split into TF32 head and remainder, zero outside the front / chunk; one
        // 16-byte row segment per thread, eight consecutive threads filling one 128-byte
        // core matrix (conflict-free shared stores)
        for (int e = tid; e < kTcM * (kBigNB / 4); e += blockDim.x) {
            const int rin = e & 7, kq = (e >> 3) & (kBigNB / 4 - 1), rg = e >> 7;
            const int r = rg * 8 + rin, k = kq * 4;
            float4 av = make_float4(0.f, 0.f, 0.f, 0.f), bv = av;
            if (k < kn && r0 + r < f) av = *(const float4*)(Lr + (int64_t)(r0 + r) * ldw + kc + k);
            if (k < kn && c0 + r < f) bv = *(const float4*)(W + (int64_t)(c0 + r) * ldw + kc + k);
            const float* ap = &av.x;
            const float* bp = &bv.x;
            float4 ah, al, bh, bl;
            float* ahp = &ah.x; float* alp = &al.x; float* bhp = &bh.x; float* blp = &bl.x;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = k + u < kn;
                const float x = in ? ap[u] : 0.0f, y = in ? bp[u] : 0.0f;
                ahp[u] = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
                alp[u] = x - ahp[u];
                bhp[u] = __uint_as_float(__float_as_uint(y) & 0xffffe000u);
                blp[u] = y - bhp[u];
            }
            const int o = ((rg * (kBigNB / 4) + kq) << 7) + (rin << 4);
            *(float4*)(Ahi + o) = ah;
            *(float4*)(Alo + o) = al;
            *(float4*)(Bhi + o) = bh;
            *(float4*)(Blo + o) = bl;
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        tmem = tmem_base;
        if (tid == 0) {
            const unsigned char* As[3] = {Ahi, Ahi, Alo};
            const unsigned char* Bs[3] = {Bhi, Blo, Bhi};
            for (int kk = 0; kk < kn; kk += 8)
                for (int q = 0; q < 3; ++q) {
                    const uint64_t ad = umma_sdesc(smem_u32(As[q]) + (kk / 4) * 128);
                    const uint64_t bd = umma_sdesc(smem_u32(Bs[q]) + (kk / 4) * 128);
                    const uint32_t acc = (kc > 0 || kk > 0 || q > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
        }
        // bounded wait for this chunk's MMAs (mbarrier phase = round parity); the staged
        // operands may only be overwritten after it
        uint32_t done = 0;
        for (int it = 0; it < (1 << 24) && !done; ++it)
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(smem_u32(&mbar)), "r"((uint32_t)(round & 1)));
        asm volatile("tcgen05.fence::after_thread_sync;");
        ok = __syncthreads_and(done) != 0;
        if (!ok) break;
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    if (ok) {
        // warp w reads the tensor-memory lanes of its quarter (w mod 4) and the 32 columns
        // of chunk w / 4
        const int quarter = warp & 3, cb = (warp >> 2) * 32;
        const int i = r0 + quarter * 32 + lane;
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cb;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
              "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
              "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (i < f) {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
                const int j = c0 + cb + jj;
                if (j < f && i >= j) F[(int64_t)j * f + i] -= __uint_as_float(v[jj]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTcM));
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
            k_big_l21x<T><<<(unsigned)((rows + 7) / 8), 128, 0, st>>>(s, k0, nb, a, F, W, nullptr, kBigNB, X);
            launches += 1 + launch_trailing<T>(s, k0, nb, rows, f, a, F, W, kBigNB, f, st);
        }
    } else {
        // FP32: outer panels of kOuterNB columns made of 64-column inner panels; an inner
        // panel updates only the rest of its outer panel (CUDA cores), and the trailing
        // matrix takes one rank-kOuterNB update on the tensor cores (3×TF32)
        T* Lr = W + (int64_t)P.max_big_f * kOuterNB;
        for (int k0 = 0; k0 < c; k0 += kOuterNB) {
            const int nbo = std::min(kOuterNB, c - k0);
            for (int k1 = k0; k1 < k0 + nbo; k1 += kBigNB) {
                const int nb = std::min(kBigNB, k0 + nbo - k1);
                k_big_diag<T><<<1, 256, 0, st>>>(s, k1, nb, a, F);
                double* X = linv + (int64_t)(k1 / kBigNB) * kBigNB * kBigNB;
                k_big_panel_inverse<T><<<kBigNB / 8, 256, 0, st>>>(s, k1, nb, a, F, X);
                const int rows = f - k1 - nb;
                launches += 2;
                if (rows <= 0) continue;
                k_big_l21x<T><<<(unsigned)((rows + 7) / 8), 128, 0, st>>>(s, k1, nb, a, F, W + (k1 - k0),
                                                                           Lr + (k1 - k0), kOuterNB, X);
                ++launches;
                const int cend = k0 + nbo;
                if (k1 + nb < cend)
                    launches += launch_trailing<T>(s, k1, nb, rows, cend, a, F, W + (k1 - k0), kOuterNB, f, st);
            }
            const int rows = f - k0 - nbo;
            if (rows > 0) {
                const int nt = (rows + kTcM - 1) / kTcM;
                k_big_trailing_tc<<<(unsigned)(nt * (nt + 1) / 2), 512, kTcSmem, st>>>(s, k0, nbo, a, F, Lr, W,
                                                                                      kOuterNB, P.big_err);
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
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_big_trailing_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    nsm();  // queried here, outside any stream capture of the launch sequences
    return 0;
}

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
