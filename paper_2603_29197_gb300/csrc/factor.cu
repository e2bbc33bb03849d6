// Numeric supernodal LDLᵀ of the permuted, statically regularised KKT matrix
// (paper §2.2: the "factor" phase, once per interior-point iteration) and the
// triangular solves (the "solve" phase, twice per iteration).
//
// Multifrontal scheme over the supernodal elimination tree, one launch per tree
// level (leaves first), one CTA per supernode s with front F_s of order f_s =
// c_s + r_s (c_s own columns, r_s rows below):
//   1. assemble F_s: the KKT entries of s's columns (read from the value array
//      through the assembly map, ±ε added on the diagonal) plus the update
//      matrices of s's children scattered through their relative indices
//      (extend-add; children are gathered by their parent, so no atomics);
//   2. dense right-looking partial LDLᵀ of the first c_s columns; a pivot whose
//      signed value is below the threshold is replaced (dynamic regularisation);
//   3. the trailing r_s×r_s block is the Schur complement (update matrix) that the
//      parent gathers.
// The front lives in shared memory while it is being factored (f_s ≤ kSmemFront)
// and is written to its slot of the front array afterwards; larger fronts are
// factored in place in global memory.  Columns 0..c_s−1 of the stored front hold
// L (unit diagonal implied) with D on the diagonal.
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
// one-thread fronts (f ≤ kThreadFront): the front lives in the thread's local array
// (column-major, leading dimension kThreadFront); used for the many tiny fronts at the
// bottom of the tree, where a warp per front would leave most FP64 lanes idle
// ---------------------------------------------------------------------------
__device__ __forceinline__ void thread_factor_front(int s, const FactorView& a, const double* __restrict__ kval) {
    constexpr int LD = kThreadFront;
    double F[LD * LD];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    for (int j = 0; j < f; ++j)
        for (int i = j; i < f; ++i) F[j * LD + i] = 0.0;
    for (int64_t e = a.amap_ptr[s]; e < a.amap_ptr[s + 1]; ++e) {
        const int off = a.amap_off[e];
        const int col = off / f, row = off - col * f;
        double v = kval[a.amap_slot[e]];
        if (row == col) v += a.dsign[first + col] > 0 ? a.eps : -a.eps;
        F[col * LD + row] = v;
    }
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int fc = a.nrow[ch], cc = a.ncol[ch], r = fc - cc;
        const double* U = a.front + a.front_off[ch] + (int64_t)cc * fc + cc;
        const int* rel = a.rel + a.upd_off[ch];
        for (int j = 0; j < r; ++j)
            for (int i = j; i < r; ++i) F[rel[j] * LD + rel[i]] += U[j * fc + i];
    }
    int nreg = 0;
    for (int k = 0; k < c; ++k) {
        double d = F[k * LD + k], inv;
        pivot(a, first + k, d, inv, nreg);
        F[k * LD + k] = d;
        a.dinv[first + k] = inv;
        // rows from the bottom up, so F(j,k) with j < i is still unscaled when row i uses it
        for (int i = f - 1; i > k; --i) {
            const double li = F[k * LD + i] * inv;
            for (int j = k + 1; j <= i; ++j) F[j * LD + i] -= li * F[k * LD + j];
            F[k * LD + i] = li;
        }
    }
    double* G = a.front + a.front_off[s];
    for (int j = 0; j < f; ++j)
        for (int i = 0; i < f; ++i) G[j * f + i] = i >= j ? F[j * LD + i] : 0.0;
    if (nreg) atomicAdd(a.nreg, nreg);
}

__device__ __forceinline__ void thread_fwd_front(int s, const FactorView& a, const double* __restrict__ rhs,
                                                 double* __restrict__ w) {
    double v[kThreadFront];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    for (int i = 0; i < f; ++i) v[i] = i < c ? rhs[a.perm[first + i]] : 0.0;
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int r = a.nrow[ch] - a.ncol[ch];
        const int* rel = a.rel + a.upd_off[ch];
        const double* u = a.upd + a.upd_off[ch];
        for (int i = 0; i < r; ++i) v[rel[i]] += u[i];
    }
    const double* L = a.front + a.front_off[s];
    for (int k = 0; k < c; ++k) {
        const double xk = v[k];
        for (int i = k + 1; i < f; ++i) v[i] -= L[k * f + i] * xk;
    }
    for (int i = 0; i < c; ++i) w[first + i] = v[i] * a.dinv[first + i];
    double* u = a.upd + a.upd_off[s];
    for (int i = c; i < f; ++i) u[i - c] = v[i];
}

__device__ __forceinline__ void thread_bwd_front(int s, const FactorView& a, const double* __restrict__ w,
                                                 double* __restrict__ xp, double* __restrict__ x, int accumulate) {
    double v[kThreadFront];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int* R = a.rows + a.row_ptr[s];
    for (int i = 0; i < f; ++i) v[i] = i < c ? w[first + i] : xp[R[i]];
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
}

__global__ void __launch_bounds__(128) k_thread_factor(const int* __restrict__ list, int n, FactorView a,
                                                       const double* __restrict__ kval) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) thread_factor_front(list[t], a, kval);
}
__global__ void __launch_bounds__(128) k_thread_fwd(const int* __restrict__ list, int n, FactorView a,
                                                    const double* __restrict__ rhs, double* __restrict__ w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) thread_fwd_front(list[t], a, rhs, w);
}
__global__ void __launch_bounds__(128) k_thread_bwd(const int* __restrict__ list, int n, FactorView a,
                                                    const double* __restrict__ w, double* __restrict__ xp,
                                                    double* __restrict__ x, int accumulate) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) thread_bwd_front(list[t], a, w, xp, x, accumulate);
}


// One CTA per front.  Dynamic shared memory: the front (f² doubles, SMEM variant) plus the
// scaled pivot column (f doubles) and the broadcast pivot reciprocal.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_front_factor(const int* __restrict__ list, FactorView a,
                                                      const double* __restrict__ kval) {
    extern __shared__ double smem[];
    const int s = list[blockIdx.x];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    double* G = a.front + a.front_off[s];
    double* F = SMEM ? smem : G;
    double* lk = SMEM ? smem + (size_t)f * f : smem;
    double* bc = lk + f;  // [0] = 1/d of the current column
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t ff = (int64_t)f * f;

    for (int64_t i = tid; i < ff; i += nt) F[i] = 0.0;
    __syncthreads();
    for (int64_t e = a.amap_ptr[s] + tid; e < a.amap_ptr[s + 1]; e += nt) {
        const int off = a.amap_off[e];
        double v = kval[a.amap_slot[e]];
        const int col = off / f, row = off - col * f;
        if (row == col) v += a.dsign[first + col] > 0 ? a.eps : -a.eps;
        F[off] = v;
    }
    __syncthreads();
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int fc = a.nrow[ch], cc = a.ncol[ch], r = fc - cc;
        const double* U = a.front + a.front_off[ch] + (int64_t)cc * fc + cc;
        const int* rel = a.rel + a.upd_off[ch];
        const int T = r * (r + 1) / 2;
        for (int t = tid; t < T; t += nt) {
            int i, j;
            tri_index(t, r, i, j);
            F[(int64_t)rel[j] * f + rel[i]] += U[(int64_t)j * fc + i];
        }
        __syncthreads();
    }
    int nreg = 0;
    double* dinv = a.dinv + first;
    for (int k = 0; k < c; ++k) {
        double* colk = F + (int64_t)k * f;
        if (tid == 0) {
            double d = colk[k], inv;
            pivot(a, first + k, d, inv, nreg);
            colk[k] = d;
            dinv[k] = inv;
            bc[0] = inv;
        }
        __syncthreads();
        const double inv = bc[0];
        const int m = f - k - 1;
        for (int i = k + 1 + tid; i < f; i += nt) lk[i] = colk[i] * inv;
        __syncthreads();
        const int T = m * (m + 1) / 2;
        for (int t = tid; t < T; t += nt) {
            int ii, jj;
            tri_index(t, m, ii, jj);
            const int i = k + 1 + ii, j = k + 1 + jj;
            F[(int64_t)j * f + i] -= lk[i] * colk[j];
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < f; i += nt) colk[i] = lk[i];
        __syncthreads();
    }
    if (tid == 0 && nreg) atomicAdd(a.nreg, nreg);
    if (SMEM)
        for (int64_t i = tid; i < ff; i += nt) G[i] = F[i];
}

// Forward solve L u = b and diagonal scaling w = D⁻¹u, one CTA per supernode of the
// level; b is read in the original order through the permutation; the update vector
// of each supernode (its below-rows' partial sums) is left for the parent.
__global__ void __launch_bounds__(128) k_fwd(const int* __restrict__ list, FactorView a,
                                             const double* __restrict__ rhs, double* __restrict__ w) {
    extern __shared__ double v[];
    const int s = list[blockIdx.x];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < f; i += nt) v[i] = i < c ? rhs[a.perm[first + i]] : 0.0;
    __syncthreads();
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int r = a.nrow[ch] - a.ncol[ch];
        const int* rel = a.rel + a.upd_off[ch];
        const double* u = a.upd + a.upd_off[ch];
        for (int i = tid; i < r; i += nt) v[rel[i]] += u[i];
        __syncthreads();
    }
    const double* L = a.front + a.front_off[s];
    for (int k = 0; k < c; ++k) {
        const double xk = v[k];
        const double* colk = L + (int64_t)k * f;
        for (int i = k + 1 + tid; i < f; i += nt) v[i] -= colk[i] * xk;
        __syncthreads();
    }
    for (int i = tid; i < c; i += nt) w[first + i] = v[i] * a.dinv[first + i];
    double* u = a.upd + a.upd_off[s];
    for (int i = c + tid; i < f; i += nt) u[i - c] = v[i];
}

// Backward solve Lᵀ x = w, parents first: the rows below a supernode are its
// ancestors' (already final) solution entries.  Writes the permuted solution xp and
// x[perm] (overwriting, or adding when accumulate != 0).
__global__ void __launch_bounds__(128) k_bwd(const int* __restrict__ list, FactorView a,
                                             const double* __restrict__ w, double* __restrict__ xp,
                                             double* __restrict__ x, int accumulate) {
    extern __shared__ double v[];
    const int s = list[blockIdx.x];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int* R = a.rows + a.row_ptr[s];
    for (int i = tid; i < f; i += nt) v[i] = i < c ? w[first + i] : xp[R[i]];
    __syncthreads();
    const double* L = a.front + a.front_off[s];
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    // contributions of the rows below: v_k −= Σ_{i ≥ c} L_ik x_i
    for (int k = wid; k < c; k += nw) {
        const double* colk = L + (int64_t)k * f;
        double acc = 0.0;
        for (int i = c + lane; i < f; i += 32) acc += colk[i] * v[i];
        acc = warp_sum(acc);
        if (lane == 0) v[k] -= acc;
    }
    __syncthreads();
    // the c×c unit upper-triangular part, sequential in k (warp 0)
    if (wid == 0) {
        for (int k = c - 1; k >= 0; --k) {
            const double* colk = L + (int64_t)k * f;
            double acc = 0.0;
            for (int i = k + 1 + lane; i < c; i += 32) acc += colk[i] * v[i];
            acc = warp_sum(acc);
            if (lane == 0) v[k] -= acc;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = tid; i < c; i += nt) {
        const double xi = v[i];
        xp[first + i] = xi;
        if (accumulate) x[a.perm[first + i]] += xi;
        else x[a.perm[first + i]] = xi;
    }
}

// ---------------------------------------------------------------------------
// warp-level variants for fronts of order ≤ kWarpFront (one warp per front, the front
// in the warp's slice of shared memory, __syncwarp instead of block barriers)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_factor_front(int s, const FactorView& a, const double* __restrict__ kval,
                                                  double* F, double* lk, int lane) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int ff = f * f;
    for (int i = lane; i < ff; i += 32) F[i] = 0.0;
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
                off[u] = eu < e1 ? a.amap_off[eu] : -1;
                v[u] = eu < e1 ? kval[a.amap_slot[eu]] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (off[u] < 0) continue;
                const int col = off[u] / f, row = off[u] - col * f;
                if (row == col) v[u] += a.dsign[first + col] > 0 ? a.eps : -a.eps;
                F[off[u]] = v[u];
            }
        }
    }
    __syncwarp();
    // extend-add of each child's update block, its lower triangle spread over the lanes
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int fc = a.nrow[ch], cc = a.ncol[ch], r = fc - cc;
        const double* U = a.front + a.front_off[ch] + (int64_t)cc * fc + cc;
        const int* rel = a.rel + a.upd_off[ch];
        const int T = r * (r + 1) / 2;
        for (int t = lane; t < T; t += 32) {
            int i, j;
            tri_index(t, r, i, j);
            F[rel[j] * f + rel[i]] += U[(int64_t)j * fc + i];
        }
        __syncwarp();
    }
    // right-looking partial LDLᵀ of the first c columns
    int nreg = 0;
    double* dinv = a.dinv + first;
    for (int k = 0; k < c; ++k) {
        double* colk = F + k * f;
        double d = 0.0, inv = 0.0;
        if (lane == 0) {
            d = colk[k];
            pivot(a, first + k, d, inv, nreg);
            colk[k] = d;
            dinv[k] = inv;
        }
        inv = __shfl_sync(0xffffffffu, inv, 0);
        const int m = f - k - 1;
        for (int i = k + 1 + lane; i < f; i += 32) lk[i] = colk[i] * inv;
        __syncwarp();
        const int T = m * (m + 1) / 2;
        for (int t = lane; t < T; t += 32) {
            int ii, jj;
            tri_index(t, m, ii, jj);
            const int i = k + 1 + ii, j = k + 1 + jj;
            F[j * f + i] -= lk[i] * colk[j];
        }
        __syncwarp();
        for (int i = k + 1 + lane; i < f; i += 32) colk[i] = lk[i];
        __syncwarp();
    }
    double* G = a.front + a.front_off[s];
    for (int i = lane; i < ff; i += 32) G[i] = F[i];
    if (lane == 0 && nreg) atomicAdd(a.nreg, nreg);
    __syncwarp();
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

__device__ __forceinline__ void warp_fwd_front(int s, const FactorView& a, const double* __restrict__ rhs,
                                               double* __restrict__ w, double* v, double* P, int lane) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    warp_load_panel(a.front + a.front_off[s], f * c, P, lane);
    for (int i = lane; i < f; i += 32) v[i] = i < c ? rhs[a.perm[first + i]] : 0.0;
    __syncwarp();
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int r = a.nrow[ch] - a.ncol[ch];
        const int* rel = a.rel + a.upd_off[ch];
        const double* u = a.upd + a.upd_off[ch];
        for (int i = lane; i < r; i += 32) v[rel[i]] += u[i];
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
}

// Column-oriented backward solve: each known x_i (i ≥ c first, then i = c−1 … 1) is
// subtracted from the own-column entries v_k, k < i, one lane per k (no reductions).
__device__ __forceinline__ void warp_bwd_front(int s, const FactorView& a, const double* __restrict__ w,
                                               double* __restrict__ xp, double* __restrict__ x, int accumulate,
                                               double* v, double* P, int lane) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int* R = a.rows + a.row_ptr[s];
    warp_load_panel(a.front + a.front_off[s], f * c, P, lane);
    for (int i = lane; i < f; i += 32) v[i] = i < c ? w[first + i] : xp[R[i]];
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
}

// one warp per subtree task (children before parents)
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_task_factor(const int* __restrict__ task, int ntask,
                                                                    FactorView a, const double* __restrict__ kval,
                                                                    int fmax) {
    extern __shared__ double smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kWarpsPerBlock + wid;
    if (t >= ntask) return;
    double* F = smem + (size_t)wid * fmax * (fmax + 1);
    const int lo = task[2 * t], hi = task[2 * t + 1];
    for (int s = lo; s <= hi; ++s) warp_factor_front(s, a, kval, F, F + fmax * fmax, lane);
}
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_task_fwd(const int* __restrict__ task, int ntask,
                                                                 FactorView a, const double* __restrict__ rhs,
                                                                 double* __restrict__ w, int fmax) {
    extern __shared__ double smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kWarpsPerBlock + wid;
    if (t >= ntask) return;
    double* v = smem + (size_t)wid * fmax * (fmax + 1);
    const int lo = task[2 * t], hi = task[2 * t + 1];
    for (int s = lo; s <= hi; ++s) warp_fwd_front(s, a, rhs, w, v, v + fmax, lane);
}
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_task_bwd(const int* __restrict__ task, int ntask,
                                                                 FactorView a, const double* __restrict__ w,
                                                                 double* __restrict__ xp, double* __restrict__ x,
                                                                 int accumulate, int fmax) {
    extern __shared__ double smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kWarpsPerBlock + wid;
    if (t >= ntask) return;
    double* v = smem + (size_t)wid * fmax * (fmax + 1);
    const int lo = task[2 * t], hi = task[2 * t + 1];
    for (int s = hi; s >= lo; --s) warp_bwd_front(s, a, w, xp, x, accumulate, v, v + fmax, lane);
}
// one warp per listed supernode of a level
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_warp_factor(const int* __restrict__ list, int n,
                                                                    FactorView a, const double* __restrict__ kval,
                                                                    int fmax) {
    extern __shared__ double smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kWarpsPerBlock + wid;
    if (t >= n) return;
    double* F = smem + (size_t)wid * fmax * (fmax + 1);
    warp_factor_front(list[t], a, kval, F, F + fmax * fmax, lane);
}
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_warp_fwd(const int* __restrict__ list, int n,
                                                                 FactorView a, const double* __restrict__ rhs,
                                                                 double* __restrict__ w, int fmax) {
    extern __shared__ double smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kWarpsPerBlock + wid;
    if (t >= n) return;
    double* v = smem + (size_t)wid * fmax * (fmax + 1);
    warp_fwd_front(list[t], a, rhs, w, v, v + fmax, lane);
}
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_warp_bwd(const int* __restrict__ list, int n,
                                                                 FactorView a, const double* __restrict__ w,
                                                                 double* __restrict__ xp, double* __restrict__ x,
                                                                 int accumulate, int fmax) {
    extern __shared__ double smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kWarpsPerBlock + wid;
    if (t >= n) return;
    double* v = smem + (size_t)wid * fmax * (fmax + 1);
    warp_bwd_front(list[t], a, w, xp, x, accumulate, v, v + fmax, lane);
}

// ---- launchers ----------------------------------------------------------------
static int wblocks(int n) { return (n + kWarpsPerBlock - 1) / kWarpsPerBlock; }
// per warp: the front vector (fmax) and the panel (≤ fmax·fmax)
static size_t wsolve_smem(int fmax) { return (size_t)kWarpsPerBlock * fmax * (fmax + 1) * sizeof(double); }

int launch_factor(const FactorPlan& P, const FactorView& a, const double* kval, cudaStream_t st) {
    int launches = 0;
    if (P.ntasks) {
        const int fm = P.task_max_f;
        k_task_factor<<<wblocks(P.ntasks), kWarpsPerBlock * 32, wsolve_smem(fm), st>>>(
            P.d_task, P.ntasks, a, kval, fm);
        ++launches;
    }
    for (int lv = 0; lv < (int)P.levels.size(); ++lv) {
        const LevelPlan& L = P.levels[lv];
        if (L.n_thread) {
            k_thread_factor<<<(L.n_thread + 127) / 128, 128, 0, st>>>(P.d_thread + L.off_thread, L.n_thread, a, kval);
            ++launches;
        }
        if (L.n_warp) {
            const int fm = L.max_warp_f;
            k_warp_factor<<<wblocks(L.n_warp), kWarpsPerBlock * 32, wsolve_smem(fm), st>>>(
                P.d_warp + L.off_warp, L.n_warp, a, kval, fm);
            ++launches;
        }
        if (L.n_small) {
            const size_t sm = ((size_t)L.max_small * (L.max_small + 1) + 1) * sizeof(double);
            const int threads = L.max_small <= 64 ? 128 : 256;
            k_front_factor<true><<<L.n_small, threads, sm, st>>>(P.d_small + L.off_small, a, kval);
            ++launches;
        }
        if (L.n_large) {
            const size_t sm = ((size_t)L.max_cta_f + 1) * sizeof(double);
            k_front_factor<false><<<L.n_large, 256, sm, st>>>(P.d_large + L.off_large, a, kval);
            ++launches;
        }
    }
    return launches;
}

int launch_solve(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                 double* x, bool accumulate, cudaStream_t st) {
    int launches = 0;
    const int nl = (int)P.levels.size();
    const int acc = accumulate ? 1 : 0;
    if (P.ntasks) {
        k_task_fwd<<<wblocks(P.ntasks), kWarpsPerBlock * 32, wsolve_smem(P.task_max_f), st>>>(
            P.d_task, P.ntasks, a, rhs, w, P.task_max_f);
        ++launches;
    }
    for (int lv = 0; lv < nl; ++lv) {
        const LevelPlan& L = P.levels[lv];
        if (L.n_thread) {
            k_thread_fwd<<<(L.n_thread + 127) / 128, 128, 0, st>>>(P.d_thread + L.off_thread, L.n_thread, a, rhs, w);
            ++launches;
        }
        if (L.n_warp) {
            k_warp_fwd<<<wblocks(L.n_warp), kWarpsPerBlock * 32, wsolve_smem(L.max_warp_f), st>>>(
                P.d_warp + L.off_warp, L.n_warp, a, rhs, w, L.max_warp_f);
            ++launches;
        }
        if (L.n_cta) {
            k_fwd<<<L.n_cta, 128, (size_t)L.max_cta_f * sizeof(double), st>>>(P.d_cta + L.off_cta, a, rhs, w);
            ++launches;
        }
    }
    for (int lv = nl - 1; lv >= 0; --lv) {
        const LevelPlan& L = P.levels[lv];
        if (L.n_thread) {
            k_thread_bwd<<<(L.n_thread + 127) / 128, 128, 0, st>>>(P.d_thread + L.off_thread, L.n_thread, a, w, xp, x,
                                                                  acc);
            ++launches;
        }
        if (L.n_warp) {
            k_warp_bwd<<<wblocks(L.n_warp), kWarpsPerBlock * 32, wsolve_smem(L.max_warp_f), st>>>(
                P.d_warp + L.off_warp, L.n_warp, a, w, xp, x, acc, L.max_warp_f);
            ++launches;
        }
        if (L.n_cta) {
            k_bwd<<<L.n_cta, 128, (size_t)L.max_cta_f * sizeof(double), st>>>(P.d_cta + L.off_cta, a, w, xp, x, acc);
            ++launches;
        }
    }
    if (P.ntasks) {
        k_task_bwd<<<wblocks(P.ntasks), kWarpsPerBlock * 32, wsolve_smem(P.task_max_f), st>>>(
            P.d_task, P.ntasks, a, w, xp, x, acc, P.task_max_f);
        ++launches;
    }
    return launches;
}

int factor_set_attributes() {
    const int warp_smem = kWarpsPerBlock * kWarpFront * (kWarpFront + 1) * (int)sizeof(double);
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_front_factor<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (kSmemFront * (kSmemFront + 1) + 1) * (int)sizeof(double)));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_front_factor<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (kMaxSolveFront + 1) * (int)sizeof(double)));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_task_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, warp_smem));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_warp_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, warp_smem));
    const int wsolve = kWarpsPerBlock * kWarpFront * (kWarpFront + 1) * (int)sizeof(double);
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_task_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, wsolve));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_task_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, wsolve));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_warp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, wsolve));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_warp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, wsolve));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSolveFront * 8));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSolveFront * 8));
    return 0;
}

}  // namespace qoco
