// Device functions of the supernodal factorisation and solves of one front (paper §2.2:
// the numeric LDLᵀ of the KKT matrix of eq. (2) and its triangular solves): one thread
// per front (order ≤ kThreadFront, the front in registers) or one warp per front (the
// front in the warp's slice of shared memory), each written as independent loads, then
// wait() (a dataflow kernel waits there for the fronts it depends on; NoWait otherwise),
// then the dependent loads and the arithmetic.  Shared by the level, dataflow and
// per-instance kernels (factor.cu) and the batched interior-point kernel (batch_ipm.cu).
#pragma once

#include "factor.h"

namespace qoco {

// Entry t of the column-major lower triangle (diagonal included) of an m×m block →
// (row ii, column jj).  Column jj starts at S(jj) = jj·m − jj(jj−1)/2.  The FP32 square
// root gives the column up to rounding; two integer checks make it exact (m ≤ 4096).
__device__ __forceinline__ void tri_index(int t, int m, int& ii, int& jj) {
    const float b = 2.0f * (float)m + 1.0f;
    int j = (int)((b - sqrtf(fmaxf(b * b - 8.0f * (float)t, 0.0f))) * 0.5f);
    j = max(0, min(j, m - 1));
    while (j > 0 && j * m - (j * (j - 1)) / 2 > t) --j;
    while (j + 1 < m && (j + 1) * m - ((j + 1) * j) / 2 <= t) ++j;
    jj = j;
    ii = t - (j * m - (j * (j - 1)) / 2) + j;
}

// F[rel_j, rel_i] += U_ij over the lower triangle of a child's r×r update block (leading
// dimension fc), spread over nt threads with four independent entries per step; the
// block was written by another thread block (read through L2).  T: the working type of
// the front (FP64; FP32 for the mixed-precision batched kernel).
template <class Real = double>
__device__ __forceinline__ void extend_add(Real* F, int f, const double* U, int fc, const int* rel, int r,
                                           int tid, int nt) {
    const int T = r * (r + 1) / 2;
    for (int t = tid; t < T; t += 4 * nt) {
        int off[4];
        double u4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int tu = t + u * nt;
            off[u] = -1;
            u4[u] = 0.0;
            if (tu < T) {
                int i, j;
                tri_index(tu, r, i, j);
                off[u] = rel[j] * f + rel[i];
                u4[u] = __ldcg(U + (int64_t)j * fc + i);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (off[u] >= 0) F[off[u]] += (Real)u4[u];
    }
}

// reciprocal in the front's working type (FP64: two Newton steps from the approximate
// reciprocal; FP32: the correctly rounded reciprocal)
__device__ __forceinline__ double rcp_w(double d) { return recip(d); }
__device__ __forceinline__ float rcp_w(float d) { return __frcp_rn(d); }

// Pivot of column k (dynamic regularisation) and its reciprocal: computed once by the
// calling thread; the caller broadcasts.  FP64 work on GB300 is scarce, so nothing is
// recomputed per lane.
__device__ __forceinline__ void pivot(const FactorView& a, int col, double& d, double& inv, int& nreg) {
    const bool pos = a.dsign[col] > 0;
    const bool ok = pos ? (d >= a.dyn_thresh) : (d <= -a.dyn_thresh);
    if (!ok) { d = pos ? a.dyn_value : -a.dyn_value; ++nreg; }
    inv = recip(d);
}


// ---------------------------------------------------------------------------
// Blocked right-looking partial LDLᵀ of the first c columns of the front F (order f,
// column-major, lower triangle), shared by the warp (NT = 32, __syncwarp) and the CTA
// (__syncthreads) kernels.  Panels of kPanel columns: each panel is factored column by
// column (pivot and its reciprocal by thread 0, broadcast through bc[0]), its unscaled
// columns are kept in W (W[i·kPanel + p] = d_p·l_ip), then the trailing lower triangle
// is updated by one rank-kPanel pass F_ij −= Σ_p l_ip·W_jp whose entries are spread
// over the threads with incrementally advanced (row, column) indices.
// ---------------------------------------------------------------------------
constexpr int kPanel = 4;

template <bool WARP>
__device__ __forceinline__ void group_sync() {
    if constexpr (WARP) __syncwarp();
    else __syncthreads();
}

// first entry t0 of the column-major lower triangle of an m×m block handled by a thread
// and the advance by `stride` entries
__device__ __forceinline__ void tri_advance(int m, int stride, int& ii, int& jj) {
    ii += stride;
    while (ii >= m && jj < m) {
        ii = ii - m + jj + 1;
        ++jj;
    }
}

// bc: broadcast slots bc[0..kPanel] (reciprocal pivots of the current panel's
// columns), then the pivot signs of the front's c columns (bc[kPanel+1 ..]), loaded in
// one parallel pass so that no pivot waits on a global load.
//
// GB300 runs a dependent FP64 FMA in ~64 cycles, so the panel step is arranged around
// its serial pivot chain.  Within a panel the columns stay unscaled; thread t owns rows
// k+1+t (+nt …), so thread 0 owns row k+1 and, as soon as it has applied column k to
// its own diagonal entry, computes the next pivot and its reciprocal while the other
// threads apply column k to their rows: one barrier per column.  At the end of the
// panel the columns are scaled in place (L) and their unscaled copy kept in W, then the
// trailing rank-kPanel update gives each thread four independent entries per step.
template <bool WARP, class Real = double>
__device__ __forceinline__ int blocked_ldlt(Real* F, Real* W, Real* bc, int f, int c, int first,
                                            const FactorView& a, int tid, int nt) {
    int nreg = 0;
    double* dinv = a.dinv + first;
    Real* sgn = bc + kPanel + 1;
    for (int k = tid; k < c; k += nt) sgn[k] = a.dsign[first + k] > 0 ? Real(1) : Real(-1);
    group_sync<WARP>();
    auto do_pivot = [&](int k) {  // thread 0 only
        Real* colk = F + (size_t)k * f;
        Real d = colk[k];
        const bool pos = sgn[k] > Real(0);
        const bool ok = pos ? (d >= (Real)a.dyn_thresh) : (d <= -(Real)a.dyn_thresh);
        if (!ok) { d = pos ? (Real)a.dyn_value : -(Real)a.dyn_value; ++nreg; }
        const Real inv = rcp_w(d);
        colk[k] = d;
        dinv[k] = sizeof(Real) == 8 ? (double)inv : recip((double)d);
        bc[k % kPanel] = inv;
    };
    if (tid == 0 && c > 0) do_pivot(0);
    for (int k0 = 0; k0 < c; k0 += kPanel) {
        const int nb = min(kPanel, c - k0);
        for (int p = 0; p < nb; ++p) {
            const int k = k0 + p;
            group_sync<WARP>();  // pivot k and column k final
            const Real* colk = F + (size_t)k * f;
            const Real inv = bc[k % kPanel];
            const int jend = k0 + nb;  // later columns of this panel: k+1 .. jend−1
            for (int i = k + 1 + tid; i < f; i += nt) {
                const Real l = colk[i] * inv;
                for (int j = k + 1; j < jend && j <= i; ++j) F[(size_t)j * f + i] -= l * colk[j];
                if (i == k + 1 && k + 1 < jend) do_pivot(k + 1);  // i == k+1 only for tid 0
            }
        }
        group_sync<WARP>();
        // scale the panel's columns (L) and keep their unscaled values in W
        for (int p = 0; p < nb; ++p) {
            const int k = k0 + p;
            Real* colk = F + (size_t)k * f;
            const Real inv = bc[k % kPanel];
            for (int i = k + 1 + tid; i < f; i += nt) {
                const Real v = colk[i];
                W[i * kPanel + p] = v;
                colk[i] = v * inv;
            }
        }
        group_sync<WARP>();
        // trailing rank-nb update of rows/columns k0+nb .. f−1, four entries per thread
        const int base = k0 + nb, m = f - base;
        if (m > 0) {
            const Real* L0 = F + (size_t)k0 * f;
            const int T = m * (m + 1) / 2;
            for (int t = tid; t < T; t += 4 * nt) {
                int ii[4], jj[4];
                Real acc[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int tu = t + u * nt;
                    if (tu < T) tri_index(tu, m, ii[u], jj[u]);
                    else { ii[u] = 0; jj[u] = 0; }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = base + ii[u], j = base + jj[u];
                    const Real* wr = W + j * kPanel;
                    Real x = F[(size_t)j * f + i];
                    x -= L0[i] * wr[0];
                    if (nb > 1) x -= L0[f + i] * wr[1];
                    if (nb > 2) x -= L0[2 * f + i] * wr[2];
                    if (nb > 3) x -= L0[3 * f + i] * wr[3];
                    acc[u] = x;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (t + u * nt < T) F[(size_t)(base + jj[u]) * f + base + ii[u]] = acc[u];
            }
        }
        group_sync<WARP>();
        if (tid == 0 && base < c) do_pivot(base);
    }
    return nreg;
}

// ---------------------------------------------------------------------------
// one-thread fronts (f ≤ kThreadFront): the front lives in the thread's local array
// (column-major, leading dimension kThreadFront); used for the many tiny fronts at the
// bottom of the tree, where a warp per front would leave most FP64 lanes idle
// ---------------------------------------------------------------------------
// No dependency to wait for (level-synchronous callers).
struct NoWait {
    __device__ __forceinline__ bool operator()() const { return true; }
};

// The factorisation of one front: zero it and assemble the KKT entries (independent of
// other fronts), wait() (the dataflow kernel waits there for the children), then the
// extend-add of the children's update blocks (read through L2: in the dataflow kernel
// they were written in the same launch) and the partial LDLᵀ.
template <class Wait, class Real = double>
__device__ __forceinline__ bool thread_factor_front(int s, const FactorView& a, const double* __restrict__ kval,
                                                    const Wait& wait) {
    constexpr int LD = kThreadFront;
    Real F[LD * LD];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    for (int j = 0; j < f; ++j)
        for (int i = j; i < f; ++i) F[j * LD + i] = Real(0);
    for (int64_t e = a.amap_ptr[s]; e < a.amap_ptr[s + 1]; ++e) {
        const int off = (int)a.amap_off[e];
        const int col = off / f, row = off - col * f;
        double v = kval[a.amap_slot[e]];
        if (row == col) v += a.dsign[first + col] > 0 ? a.eps : -a.eps;
        F[col * LD + row] = (Real)v;
    }
    if (!wait()) return false;
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int fc = a.nrow[ch], cc = a.ncol[ch], r = fc - cc;
        const double* U = a.front + a.front_off[ch] + (int64_t)cc * fc + cc;
        const int* rel = a.rel + a.upd_off[ch];
        for (int j = 0; j < r; ++j)
            for (int i = j; i < r; ++i) F[rel[j] * LD + rel[i]] += (Real)__ldcg(U + j * fc + i);
    }
    int nreg = 0;
    for (int k = 0; k < c; ++k) {
        Real inv;
        if constexpr (sizeof(Real) == 8) {
            double d = F[k * LD + k], dinv;
            pivot(a, first + k, d, dinv, nreg);
            F[k * LD + k] = d;
            a.dinv[first + k] = dinv;
            inv = dinv;
        } else {
            Real d = F[k * LD + k];
            const bool pos = a.dsign[first + k] > 0;
            const bool ok = pos ? (d >= (Real)a.dyn_thresh) : (d <= -(Real)a.dyn_thresh);
            if (!ok) { d = pos ? (Real)a.dyn_value : -(Real)a.dyn_value; ++nreg; }
            F[k * LD + k] = d;
            a.dinv[first + k] = recip((double)d);
            inv = rcp_w(d);
        }
        // rows from the bottom up, so F(j,k) with j < i is still unscaled when row i uses it
        for (int i = f - 1; i > k; --i) {
            const Real li = F[k * LD + i] * inv;
            for (int j = k + 1; j <= i; ++j) F[j * LD + i] -= li * F[k * LD + j];
            F[k * LD + i] = li;
        }
    }
    double* G = a.front + a.front_off[s];
    for (int j = 0; j < f; ++j)
        for (int i = 0; i < f; ++i) G[j * f + i] = i >= j ? (double)F[j * LD + i] : 0.0;
    if (nreg) atomicAdd(a.nreg, nreg);
    return true;
}

// The solve steps of one front are written as: loads that do not depend on other
// fronts, then wait() (the dataflow kernel waits there for the fronts this one depends
// on), then the dependent loads and the arithmetic.  Results of other fronts are read
// through L2 (__ldcg): in the dataflow kernel they were written in the same launch.
template <class Wait>
__device__ __forceinline__ bool thread_fwd_front(int s, const FactorView& a, const double* __restrict__ rhs,
                                                 double* __restrict__ w, const Wait& wait) {
    double v[kThreadFront];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    for (int i = 0; i < f; ++i) v[i] = i < c ? rhs[a.perm[first + i]] : 0.0;
    if (!wait()) return false;
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int r = a.nrow[ch] - a.ncol[ch];
        const int* rel = a.rel + a.upd_off[ch];
        const double* u = a.upd + a.upd_off[ch];
        for (int i = 0; i < r; ++i) v[rel[i]] += __ldcg(u + i);
    }
    const double* L = a.front + a.front_off[s];
    for (int k = 0; k < c; ++k) {
        const double xk = v[k];
        for (int i = k + 1; i < f; ++i) v[i] -= L[k * f + i] * xk;
    }
    for (int i = 0; i < c; ++i) w[first + i] = v[i] * a.dinv[first + i];
    double* u = a.upd + a.upd_off[s];
    for (int i = c; i < f; ++i) u[i - c] = v[i];
    return true;
}

template <class Wait>
__device__ __forceinline__ bool thread_bwd_front(int s, const FactorView& a, const double* __restrict__ w,
                                                 double* __restrict__ xp, double* __restrict__ x, int accumulate,
                                                 const Wait& wait) {
    double v[kThreadFront];
    int R[kThreadFront];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int* Rg = a.rows + a.row_ptr[s];
    for (int i = c; i < f; ++i) R[i] = Rg[i];
    if (!wait()) return false;
    for (int i = 0; i < f; ++i) v[i] = __ldcg(i < c ? w + first + i : xp + R[i]);
    const double* L = a.front + a.front_off[s];
    for (int k = c - 1; k >= 0; --k) {
        double acc = v[k];
        for (int i = k + 1; i < f; ++i) acc -= L[k * f + i] * v[i];
        v[k] = acc;
    }
    for (int i = 0; i < c; ++i) {
        xp[first + i] = v[i];
        if (accumulate) x[a.perm[first + i]] += v[i];
        else x[a.perm[first + i]] = v[i];
    }
    return true;
}

// per-warp shared memory of the warp factor kernels: front (fmax²), W panel (kPanel·fmax)
// and the broadcast slot
__host__ __device__ constexpr int wfactor_stride(int fmax) { return fmax * (fmax + kPanel) + kPanel + 1 + fmax; }

// ---------------------------------------------------------------------------
// warp-level variants for fronts of order ≤ kWarpFront (one warp per front, the front
// in the warp's slice of shared memory, __syncwarp instead of block barriers)
// ---------------------------------------------------------------------------
template <class Wait, class Real = double>
__device__ __forceinline__ bool warp_factor_front(int s, const FactorView& a, const double* __restrict__ kval,
                                                  Real* F, Real* lk, int lane, const Wait& wait) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int ff = f * f;
    for (int i = lane; i < ff; i += 32) F[i] = Real(0);
    __syncwarp();
    // original entries (static regularisation on the diagonal): loads first, then stores
    {
        const int64_t e0 = a.amap_ptr[s], e1 = a.amap_ptr[s + 1];
        for (int64_t e = e0 + lane; e < e1; e += 4 * 32) {
            int off[4];
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t eu = e + u * 32;
                off[u] = eu < e1 ? (int)a.amap_off[eu] : -1;
                v[u] = eu < e1 ? kval[a.amap_slot[eu]] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (off[u] < 0) continue;
                const int col = off[u] / f, row = off[u] - col * f;
                if (row == col) v[u] += a.dsign[first + col] > 0 ? a.eps : -a.eps;
                F[off[u]] = (Real)v[u];
            }
        }
    }
    // child records of the first 32 children, one per lane (loaded before the wait)
    const int k0 = a.child_ptr[s], nch = a.child_ptr[s + 1] - k0;
    ChildInfo mine;
    if (lane < nch) mine = a.cinfo[k0 + lane];
    __syncwarp();
    if (!wait()) return false;
    // extend-add of each child's update block, its lower triangle spread over the lanes
    for (int k = 0; k < nch; ++k) {
        ChildInfo ci;
        if (k < 32) {
            ci.u_off = __shfl_sync(0xffffffffu, mine.u_off, k);
            ci.rel_off = __shfl_sync(0xffffffffu, mine.rel_off, k);
            ci.fc = __shfl_sync(0xffffffffu, mine.fc, k);
            ci.r = __shfl_sync(0xffffffffu, mine.r, k);
        } else {
            ci = a.cinfo[k0 + k];
        }
        const double* U = a.front + ci.u_off;
        const int* rel = a.rel + ci.rel_off;
        const int r = ci.r, fc = ci.fc;
        extend_add<Real>(F, f, U, fc, rel, r, lane, 32);
        __syncwarp();
    }
    const int nreg = blocked_ldlt<true, Real>(F, lk, lk + kPanel * f, f, c, first, a, lane, 32);
    double* G = a.front + a.front_off[s];
    for (int i = lane; i < ff; i += 32) G[i] = (double)F[i];
    if (lane == 0 && nreg) atomicAdd(a.nreg, nreg);
    __syncwarp();
    return true;
}

// copy the f×c panel of supernode s (L and D) into shared memory with independent loads
__device__ __forceinline__ void warp_load_panel(const double* __restrict__ L, int n, double* P, int lane) {
    int i = lane;
    for (; i + 3 * 32 < n; i += 4 * 32) {
        const double a0 = L[i], a1 = L[i + 32], a2 = L[i + 64], a3 = L[i + 96];
        P[i] = a0; P[i + 32] = a1; P[i + 64] = a2; P[i + 96] = a3;
    }
    for (; i < n; i += 32) P[i] = L[i];
}

template <class Wait>
__device__ __forceinline__ bool warp_fwd_front(int s, const FactorView& a, const double* __restrict__ rhs,
                                               double* __restrict__ w, double* v, double* P, int lane,
                                               const Wait& wait) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    warp_load_panel(a.front + a.front_off[s], f * c, P, lane);
    for (int i = lane; i < f; i += 32) v[i] = i < c ? rhs[a.perm[first + i]] : 0.0;
    const int k0 = a.child_ptr[s], nch = a.child_ptr[s + 1] - k0;
    ChildInfo mine;
    if (lane < nch) mine = a.cinfo[k0 + lane];
    __syncwarp();
    if (!wait()) return false;
    for (int k = 0; k < nch; ++k) {
        int64_t ro;
        int r;
        if (k < 32) {
            ro = __shfl_sync(0xffffffffu, mine.rel_off, k);
            r = __shfl_sync(0xffffffffu, mine.r, k);
        } else {
            ro = a.cinfo[k0 + k].rel_off;
            r = a.cinfo[k0 + k].r;
        }
        const int* rel = a.rel + ro;
        const double* u = a.upd + ro;
        for (int i = lane; i < r; i += 32) v[rel[i]] += __ldcg(u + i);
        __syncwarp();
    }
    for (int k = 0; k < c; ++k) {
        const double xk = v[k];
        const double* colk = P + k * f;
        for (int i = k + 1 + lane; i < f; i += 32) v[i] -= colk[i] * xk;
        __syncwarp();
    }
    const double* dinv = a.dinv + first;
    for (int i = lane; i < c; i += 32) w[first + i] = v[i] * dinv[i];
    double* u = a.upd + a.upd_off[s];
    for (int i = c + lane; i < f; i += 32) u[i - c] = v[i];
    __syncwarp();
    return true;
}

// Column-oriented backward solve: each known x_i (i ≥ c first, then i = c−1 … 1) is
// subtracted from the own-column entries v_k, k < i, one lane per k (no reductions).
template <class Wait>
__device__ __forceinline__ bool warp_bwd_front(int s, const FactorView& a, const double* __restrict__ w,
                                               double* __restrict__ xp, double* __restrict__ x, int accumulate,
                                               double* v, double* P, int lane, const Wait& wait) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int* R = a.rows + a.row_ptr[s];
    warp_load_panel(a.front + a.front_off[s], f * c, P, lane);
    const int r0 = lane < f ? R[lane] : 0, r1 = lane + 32 < f ? R[lane + 32] : 0;  // f ≤ 64
    if (!wait()) return false;
    if (lane < f) v[lane] = __ldcg(lane < c ? w + first + lane : xp + r0);
    if (lane + 32 < f) v[lane + 32] = __ldcg(lane + 32 < c ? w + first + lane + 32 : xp + r1);
    __syncwarp();
    for (int i = c; i < f; ++i) {
        const double xi = v[i];
        for (int k = lane; k < c; k += 32) v[k] -= P[k * f + i] * xi;
    }
    __syncwarp();
    for (int i = c - 1; i > 0; --i) {
        const double xi = v[i];
        for (int k = lane; k < i; k += 32) v[k] -= P[k * f + i] * xi;
        __syncwarp();
    }
    for (int i = lane; i < c; i += 32) {
        const double xi = v[i];
        xp[first + i] = xi;
        if (accumulate) x[a.perm[first + i]] += xi;
        else x[a.perm[first + i]] = xi;
    }
    __syncwarp();
    return true;
}

}  // namespace qoco
