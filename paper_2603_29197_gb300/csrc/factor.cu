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

template <bool SMEM>
__global__ void __launch_bounds__(256) k_front_factor(const int* __restrict__ list, FactorView a,
                                                      const double* __restrict__ kval) {
    extern __shared__ double smem[];
    const int s = list[blockIdx.x];
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    double* G = a.front + a.front_off[s];
    double* F = SMEM ? smem : G;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t ff = (int64_t)f * f;

    for (int64_t i = tid; i < ff; i += nt) F[i] = 0.0;
    __syncthreads();
    for (int64_t e = a.amap_ptr[s] + tid; e < a.amap_ptr[s + 1]; e += nt) {
        const int off = a.amap_off[e];
        double v = kval[a.amap_slot[e]];
        const int col = off / f, row = off - col * f;
        if (row == col) v += a.eps * (double)a.dsign[first + col];
        F[off] = v;
    }
    __syncthreads();
    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1]; ++k) {
        const int ch = a.child[k];
        const int fc = a.nrow[ch], cc = a.ncol[ch], r = fc - cc;
        const double* U = a.front + a.front_off[ch] + (int64_t)cc * fc + cc;
        const int* rel = a.rel + a.upd_off[ch];
        for (int idx = tid; idx < r * r; idx += nt) {
            const int i = idx % r, j = idx / r;
            if (i >= j) F[(int64_t)rel[j] * f + rel[i]] += U[(int64_t)j * fc + i];
        }
        __syncthreads();
    }
    int nreg = 0;
    for (int k = 0; k < c; ++k) {
        double d = F[(int64_t)k * f + k];
        const double sg = (double)a.dsign[first + k];
        if (!(sg * d >= a.dyn_thresh)) { d = sg * a.dyn_value; ++nreg; }
        const double inv = 1.0 / d;
        const int m = f - k - 1;
        const double* colk = F + (int64_t)k * f;
        for (int idx = tid; idx < m * m; idx += nt) {
            const int ii = idx % m, jj = idx / m;
            if (ii >= jj) {
                const int i = k + 1 + ii, j = k + 1 + jj;
                F[(int64_t)j * f + i] -= colk[i] * colk[j] * inv;
            }
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < f; i += nt) F[(int64_t)k * f + i] *= inv;
        if (tid == 0) F[(int64_t)k * f + k] = d;
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
    for (int i = tid; i < c; i += nt) w[first + i] = v[i] / L[(int64_t)i * f + i];
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

// ---- launchers ----------------------------------------------------------------
int launch_factor(const FactorPlan& P, const FactorView& a, const double* kval, cudaStream_t st) {
    int launches = 0;
    for (int lv = 0; lv < (int)P.levels.size(); ++lv) {
        const LevelPlan& L = P.levels[lv];
        if (L.n_small) {
            const size_t sm = (size_t)L.max_small * L.max_small * sizeof(double);
            const int threads = L.max_small <= 48 ? 128 : 256;
            k_front_factor<true><<<L.n_small, threads, sm, st>>>(P.d_small + L.off_small, a, kval);
            ++launches;
        }
        if (L.n_large) {
            k_front_factor<false><<<L.n_large, 256, 0, st>>>(P.d_large + L.off_large, a, kval);
            ++launches;
        }
    }
    return launches;
}

int launch_solve(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                 double* x, bool accumulate, cudaStream_t st) {
    int launches = 0;
    const int nl = (int)P.levels.size();
    for (int lv = 0; lv < nl; ++lv) {
        const LevelPlan& L = P.levels[lv];
        k_fwd<<<L.count, 128, (size_t)L.max_f * sizeof(double), st>>>(P.d_all + L.off_all, a, rhs, w);
        ++launches;
    }
    for (int lv = nl - 1; lv >= 0; --lv) {
        const LevelPlan& L = P.levels[lv];
        k_bwd<<<L.count, 128, (size_t)L.max_f * sizeof(double), st>>>(P.d_all + L.off_all, a, w, xp, x,
                                                                      accumulate ? 1 : 0);
        ++launches;
    }
    return launches;
}

int factor_set_attributes() {
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_front_factor<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemFront * kSmemFront * (int)sizeof(double)));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSolveFront * 8));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSolveFront * 8));
    return 0;
}

}  // namespace qoco
