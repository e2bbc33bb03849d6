// Row kernels over the full symmetric KKT (CSR, original x | y | z order): the
// interior-point residuals with their ∞-norms and dot products (K6 + K8 inputs),
// the refinement residual r − Kx, and ‖K‖∞.  A group of LPR lanes owns one row;
// each block writes its partial sums / maxima to `partial[block][·]`, and one
// single-block kernel reduces them in a fixed order (deterministic results).
#include "row_kernels.h"

namespace qoco {

constexpr int kRowThreads = 256;
constexpr int kMaxRowBlocks = 152 * 8;  // grid cap: 8 blocks (64 warps, a full SM) per SM

template <int NV>
__device__ __forceinline__ void store_partials(double (&v)[NV], const bool (&is_max)[NV], double* partial) {
    __shared__ double sm[NV * 32];
    block_reduce<NV>(v, is_max, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[(int64_t)blockIdx.x * NV + k] = v[k];
}

// Grid-stride over rows: a block of kRowThreads threads holds kRowThreads/LPR row groups;
// every lane of a block runs the same number of loop trips, so the shuffles inside
// group_sum always see full warps.  The grid is capped (kMaxRowBlocks) so that the
// single-block finalisation reduces few partials.

constexpr int kLongThreads = 512;

// residuals: r_x = Px + c + Aᵀy + Gᵀz, r_y = Ax − b, r_z = Gx + s − h
// One row's outputs from its three partial products a0 = K_row,x·x, a1 = K_row,y·y,
// a2 = K_row,z·z, accumulated into the block's sums and maxima v.
__device__ __forceinline__ void residual_row(int row, int n, int p, double a0, double a1, double a2,
                                             const double* __restrict__ xyz, const double* __restrict__ s,
                                             const double* __restrict__ c, const double* __restrict__ b,
                                             const double* __restrict__ h, double* __restrict__ r,
                                             double (&v)[kResNV]) {
    if (row < n) {
        const double rx = a0 + c[row] + a1 + a2;
        r[row] = rx;
        v[0] += xyz[row] * a0;  // xᵀPx
        v[1] += c[row] * xyz[row];
        v[5] = amax(v[5], a0);   // |Px|
        v[6] = amax(v[6], a1);   // |Aᵀy|
        v[7] = amax(v[7], a2);   // |Gᵀz|
        v[10] = amax(v[10], rx);
    } else if (row < n + p) {
        const int i = row - n;
        const double ry = a0 - b[i];
        r[row] = ry;
        v[2] += b[i] * xyz[row];
        v[8] = amax(v[8], a0);   // |Ax|
        v[11] = amax(v[11], ry);
    } else {
        const int i = row - n - p;
        const double rz = a0 + s[i] - h[i];
        r[row] = rz;
        v[3] += h[i] * xyz[row];
        v[4] += s[i] * xyz[row];
        v[9] = amax(v[9], a0);   // |Gx|
        v[12] = amax(v[12], rz);
        v[13] = amax(v[13], s[i]);
    }
}

// sums: xᵀPx, cᵀx, bᵀy, hᵀz, sᵀz   maxes: |Px|,|Aᵀy|,|Gᵀz|,|Ax|,|Gx|,|r_x|,|r_y|,|r_z|,|s|
template <int LPR>
__global__ void __launch_bounds__(kRowThreads) k_residual(KKTView K, const double* __restrict__ xyz,
                                                         const double* __restrict__ s,
                                                         const double* __restrict__ c,
                                                         const double* __restrict__ b,
                                                         const double* __restrict__ h,
                                                         double* __restrict__ r, double* partial) {
    constexpr int GPB = kRowThreads / LPR;
    const int grp = threadIdx.x / LPR, lane = threadIdx.x % LPR;
    const int n = K.n, p = K.p;
    double v[kResNV];
    bool is_max[kResNV];
#pragma unroll
    for (int k = 0; k < kResNV; ++k) { v[k] = 0.0; is_max[k] = k >= kResNSum; }
    for (int base = blockIdx.x * GPB; base < K.N; base += gridDim.x * GPB) {
        const int row = base + grp;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        bool mine = row < K.N;
        if (mine) {
            const int64_t beg = K.rowptr[row], end = K.rowptr[row + 1];
            mine = end - beg <= kLongRow;
            if (mine) {
                // a row's columns are sorted (x, then y, then z): each lane runs its x, y and z
                // entries as three straight loops, one FP64 multiply-add per entry (a per-entry
                // three-way branch made diverging lanes issue every branch's add); y and z rows
                // use only their x part
                int64_t t = beg + lane;
                for (; t < end; t += LPR) {
                    const int j = K.colidx[t];
                    if (j >= n) break;
                    a0 += K.val[t] * xyz[j];
                }
                if (row < n) {
                    for (; t < end; t += LPR) {
                        const int j = K.colidx[t];
                        if (j >= n + p) break;
                        a1 += K.val[t] * xyz[j];
                    }
                    for (; t < end; t += LPR) a2 += K.val[t] * xyz[K.colidx[t]];
                }
            }
        }
        a0 = group_sum<LPR>(a0);
        a1 = group_sum<LPR>(a1);
        a2 = group_sum<LPR>(a2);
        if (mine && lane == 0) residual_row(row, n, p, a0, a1, a2, xyz, s, c, b, h, r, v);
    }
    store_partials<kResNV>(v, is_max, partial);
}

// Sum of NV values over the whole block, in a fixed order; valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sm[NV * 32];
    bool is_sum[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) is_sum[k] = false;
    block_reduce<NV>(v, is_sum, sm);
}

// The long rows of the residual pass: block b takes row long_rows[b] and writes its
// contributions as partial block nb + b.
__global__ void __launch_bounds__(kLongThreads) k_residual_long(KKTView K, const double* __restrict__ xyz,
                                                               const double* __restrict__ s,
                                                               const double* __restrict__ c,
                                                               const double* __restrict__ b,
                                                               const double* __restrict__ h,
                                                               double* __restrict__ r, double* partial, int nb) {
    const int row = K.long_rows[blockIdx.x], n = K.n, p = K.p;
    double a[3] = {0.0, 0.0, 0.0};
    for (int64_t t = K.rowptr[row] + threadIdx.x; t < K.rowptr[row + 1]; t += kLongThreads) {
        const int j = K.colidx[t];
        const double kv = K.val[t] * xyz[j];
        if (j < n) a[0] += kv;
        else if (j < n + p) a[1] += kv;
        else a[2] += kv;
    }
    block_sum<3>(a);
    if (threadIdx.x != 0) return;
    double v[kResNV];
#pragma unroll
    for (int k = 0; k < kResNV; ++k) v[k] = 0.0;
    residual_row(row, n, p, a[0], a[1], a[2], xyz, s, c, b, h, r, v);
    for (int k = 0; k < kResNV; ++k) partial[(int64_t)(nb + blockIdx.x) * kResNV + k] = v[k];
}

// Componentwise (Oettli–Prager) backward error of one row: |res_i| / (|K||x| + |r|)_i;
// a row whose denominator is 0 counts 0 when its residual is 0, else +inf.
__device__ __forceinline__ double cw_ratio(double e, double dn) {
    return dn > 0.0 ? fabs(e) / dn : (e == 0.0 ? 0.0 : __longlong_as_double(0x7ff0000000000000LL));
}

// res = r − K x (unregularised K); maxes |res|, |x|, |r| and (CW) the componentwise
// backward error; den (optional, CW) = |K||x| + |r| per row
template <int LPR, bool CW>
__global__ void __launch_bounds__(kRowThreads) k_spmv_res(KKTView K, const double* __restrict__ x,
                                                         const double* __restrict__ r,
                                                         double* __restrict__ res, double* __restrict__ den,
                                                         double* partial) {
    constexpr int GPB = kRowThreads / LPR;
    const int grp = threadIdx.x / LPR, lane = threadIdx.x % LPR;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const bool is_max[4] = {true, true, true, true};
    for (int base = blockIdx.x * GPB; base < K.N; base += gridDim.x * GPB) {
        const int row = base + grp;
        double acc = 0.0, aac = 0.0;
        bool mine = row < K.N;
        if (mine) {
            const int64_t beg = K.rowptr[row], end = K.rowptr[row + 1];
            mine = end - beg <= kLongRow;
            if (mine)
                for (int64_t t = beg + lane; t < end; t += LPR) {
                    const double kv = K.val[t] * x[K.colidx[t]];
                    acc += kv;
                    if (CW) aac += fabs(kv);
                }
        }
        acc = group_sum<LPR>(acc);
        if (CW) aac = group_sum<LPR>(aac);
        if (mine && lane == 0) {
            const double e = r[row] - acc, dn = aac + fabs(r[row]);
            res[row] = e;
            if (CW && den) den[row] = dn;
            v[0] = amax(v[0], e);
            v[1] = amax(v[1], x[row]);
            v[2] = amax(v[2], r[row]);
            if (CW) v[3] = amax(v[3], cw_ratio(e, dn));
        }
    }
    store_partials<4>(v, is_max, partial);
}

__global__ void __launch_bounds__(kLongThreads) k_spmv_res_long(KKTView K, const double* __restrict__ x,
                                                               const double* __restrict__ r,
                                                               double* __restrict__ res, double* __restrict__ den,
                                                               double* partial, int nb) {
    const int row = K.long_rows[blockIdx.x];
    double a[2] = {0.0, 0.0};
    for (int64_t t = K.rowptr[row] + threadIdx.x; t < K.rowptr[row + 1]; t += kLongThreads) {
        const double kv = K.val[t] * x[K.colidx[t]];
        a[0] += kv;
        a[1] += fabs(kv);
    }
    block_sum<2>(a);
    if (threadIdx.x != 0) return;
    const double e = r[row] - a[0], dn = a[1] + fabs(r[row]);
    res[row] = e;
    if (den) den[row] = dn;
    double* out = partial + (int64_t)(nb + blockIdx.x) * 4;
    out[0] = fabs(e);
    out[1] = fabs(x[row]);
    out[2] = fabs(r[row]);
    out[3] = cw_ratio(e, dn);
}

// max_i Σ_j |K_ij|
template <int LPR>
__global__ void __launch_bounds__(kRowThreads) k_norm_inf(KKTView K, double* partial) {
    constexpr int GPB = kRowThreads / LPR;
    const int grp = threadIdx.x / LPR, lane = threadIdx.x % LPR;
    double v[1] = {0.0};
    const bool is_max[1] = {true};
    for (int base = blockIdx.x * GPB; base < K.N; base += gridDim.x * GPB) {
        const int row = base + grp;
        double acc = 0.0;
        if (row < K.N) {
            const int64_t beg = K.rowptr[row], end = K.rowptr[row + 1];
            if (end - beg <= kLongRow)
                for (int64_t t = beg + lane; t < end; t += LPR) acc += fabs(K.val[t]);
        }
        acc = group_sum<LPR>(acc);
        v[0] = amax(v[0], acc);
    }
    store_partials<1>(v, is_max, partial);
}

__global__ void __launch_bounds__(kLongThreads) k_norm_inf_long(KKTView K, double* partial, int nb) {
    const int row = K.long_rows[blockIdx.x];
    double a[1] = {0.0};
    for (int64_t t = K.rowptr[row] + threadIdx.x; t < K.rowptr[row + 1]; t += kLongThreads) a[0] += fabs(K.val[t]);
    block_sum<1>(a);
    if (threadIdx.x == 0) partial[nb + blockIdx.x] = a[0];
}

// one block: reduce NV columns of partial[nb][NV] in a fixed order into out[NV], one warp
// per column (lane-strided partial results, then a fixed shuffle tree), all columns at
// once; max columns compare bit patterns (non-negative values; a NaN propagates)
__device__ void reduce_columns(const double* partial, int nb, int NV, unsigned max_mask, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    for (int k = wid; k < NV; k += nw) {
        const bool mx = (max_mask >> k) & 1u;
        double a = 0.0;
        for (int i = lane; i < nb; i += 32) {
            const double t = partial[(int64_t)i * NV + k];
            if (mx) {
                const long long bt = __double_as_longlong(t), ba = __double_as_longlong(a);
                a = bt > ba ? t : a;
            } else {
                a += t;
            }
        }
        a = mx ? warp_max_nonneg(a) : warp_sum(a);
        if (lane == 0) out[k] = a;
    }
    __syncthreads();
}

__global__ void k_finalize_residual(const double* __restrict__ partial, int nb, IPMScalars* S) {
    __shared__ double red[kResNV];
    reduce_columns(partial, nb, kResNV, ((1u << kResNV) - 1) & ~((1u << kResNSum) - 1), red);
    if (threadIdx.x != 0) return;
    const double xPx = red[0], cx = red[1], by = red[2], hz = red[3], sz = red[4];
    S->pobj = 0.5 * xPx + cx;
    S->dobj = -0.5 * xPx - by - hz;
    S->gap = sz;
    S->mu = S->nu > 0 ? sz / S->nu : 0.0;
    S->Px_inf = red[5]; S->Aty_inf = red[6]; S->Gtz_inf = red[7];
    S->Ax_inf = red[8]; S->Gx_inf = red[9];
    S->rx_inf = red[10]; S->ry_inf = red[11]; S->rz_inf = red[12]; S->s_inf = red[13];
    bool finite = true;
    for (int k = 0; k < kResNV; ++k) finite = finite && isfinite(red[k]);
    S->nonfinite = finite ? 0 : 1;
    auto conv = [&](double ea, double er) {
        const bool oy = S->ry_inf <= ea + er * fmax(S->Ax_inf, S->b_inf);
        const bool oz = S->rz_inf <= ea + er * fmax(S->Gx_inf, fmax(S->s_inf, S->h_inf));
        const bool ox = S->rx_inf <= ea + er * fmax(fmax(S->Px_inf, S->Aty_inf), fmax(S->Gtz_inf, S->c_inf));
        const bool og = fabs(S->gap) <= ea + er * fmax(1.0, fmax(fabs(S->pobj), fabs(S->dobj)));
        return ox && oy && oz && og;
    };
    S->converged = conv(S->abstol, S->reltol) ? 1 : 0;
    S->converged_inacc = conv(S->abstol_inacc, S->reltol_inacc) ? 1 : 0;
}

__global__ void k_finalize_refine(const double* __restrict__ partial, int nb, IPMScalars* S) {
    __shared__ double red[4];
    reduce_columns(partial, nb, 4, 15u, red);
    if (threadIdx.x != 0) return;
    // a non-finite residual, iterate or right-hand side ends the refinement with a
    // non-finite backward error (the caller sees it and does not accept the solve)
    const bool finite = isfinite(red[0]) && isfinite(red[1]) && isfinite(red[2]);
    const double den = S->normK * red[1] + red[2];
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const double be = !finite ? nan : den > 0.0 ? red[0] / den : 0.0;
    S->berr = be;
    S->berr_cw = finite ? red[3] : nan;
    S->refine_den = den;
    S->refine_done = (!finite || be <= S->refine_tol) ? 1 : 0;
}

__global__ void k_finalize_norm(const double* __restrict__ partial, int nb, IPMScalars* S) {
    __shared__ double red[1];
    reduce_columns(partial, nb, 1, 1u, red);
    if (threadIdx.x == 0) S->normK = red[0];
}

// ---- launchers ----------------------------------------------------------------
static int rows_blocks(int N, int lpr) {
    const int rows_per_block = kRowThreads / lpr;
    const int need = (N + rows_per_block - 1) / rows_per_block;
    return need < kMaxRowBlocks ? (need > 0 ? need : 1) : kMaxRowBlocks;
}
// partial-buffer size in doubles: the most blocks (32 lanes per row) times the most
// values per block (the residual pass)
int row_partials(int N, int n_long) { return (rows_blocks(N, 32) + n_long) * kResNV; }

#define QOCO_LPR_SWITCH(lpr, KERNEL, ...)                                          \
    switch (lpr) {                                                                 \
        case 1: KERNEL<1><<<rows_blocks(K.N, 1), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 1); break;   \
        case 2: KERNEL<2><<<rows_blocks(K.N, 2), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 2); break;   \
        case 4: KERNEL<4><<<rows_blocks(K.N, 4), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 4); break;   \
        case 8: KERNEL<8><<<rows_blocks(K.N, 8), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 8); break;   \
        case 16: KERNEL<16><<<rows_blocks(K.N, 16), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 16); break; \
        default: KERNEL<32><<<rows_blocks(K.N, 32), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 32); break; \
    }

#define QOCO_LPR_SWITCH2(lpr, KERNEL, B, ...)                                                                 \
    switch (lpr) {                                                                                            \
        case 1: KERNEL<1, B><<<rows_blocks(K.N, 1), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 1); break;   \
        case 2: KERNEL<2, B><<<rows_blocks(K.N, 2), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 2); break;   \
        case 4: KERNEL<4, B><<<rows_blocks(K.N, 4), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 4); break;   \
        case 8: KERNEL<8, B><<<rows_blocks(K.N, 8), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 8); break;   \
        case 16: KERNEL<16, B><<<rows_blocks(K.N, 16), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 16); break; \
        default: KERNEL<32, B><<<rows_blocks(K.N, 32), kRowThreads, 0, st>>>(__VA_ARGS__); nb = rows_blocks(K.N, 32); break; \
    }

int launch_residual(const KKTView& K, int lpr, const double* xyz, const double* s, const double* c,
                    const double* b, const double* h, double* r, double* partial, int64_t cap,
                    IPMScalars* S, cudaStream_t st) {
    if ((int64_t)(rows_blocks(K.N, lpr) + K.n_long) * kResNV > cap) return -1;
    int nb = 0;
    QOCO_LPR_SWITCH(lpr, k_residual, K, xyz, s, c, b, h, r, partial)
    if (K.n_long) k_residual_long<<<K.n_long, kLongThreads, 0, st>>>(K, xyz, s, c, b, h, r, partial, nb);
    k_finalize_residual<<<1, 1024, 0, st>>>(partial, nb + K.n_long, S);
    return K.n_long ? 3 : 2;
}
int launch_spmv_res(const KKTView& K, int lpr, const double* x, const double* r, double* res,
                    double* partial, int64_t cap, IPMScalars* S, cudaStream_t st, bool cw, double* den) {
    if ((int64_t)(rows_blocks(K.N, lpr) + K.n_long) * 4 > cap) return -1;
    int nb = 0;
    if (cw) {
        QOCO_LPR_SWITCH2(lpr, k_spmv_res, true, K, x, r, res, den, partial)
    } else {
        QOCO_LPR_SWITCH2(lpr, k_spmv_res, false, K, x, r, res, den, partial)
    }
    if (K.n_long) k_spmv_res_long<<<K.n_long, kLongThreads, 0, st>>>(K, x, r, res, den, partial, nb);
    k_finalize_refine<<<1, 1024, 0, st>>>(partial, nb + K.n_long, S);
    return K.n_long ? 3 : 2;
}
int launch_norm_inf(const KKTView& K, int lpr, double* partial, int64_t cap, IPMScalars* S,
                    cudaStream_t st) {
    if ((int64_t)(rows_blocks(K.N, lpr) + K.n_long) > cap) return -1;
    int nb = 0;
    QOCO_LPR_SWITCH(lpr, k_norm_inf, K, partial)
    if (K.n_long) k_norm_inf_long<<<K.n_long, kLongThreads, 0, st>>>(K, partial, nb);
    k_finalize_norm<<<1, 1024, 0, st>>>(partial, nb + K.n_long, S);
    return K.n_long ? 3 : 2;
}

}  // namespace qoco
