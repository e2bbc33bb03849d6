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

// barrier of the group that works on one front: its warp (or the lanes of `mask`, when a
// warp holds several fronts) or its CTA
template <bool WARP>
__device__ __forceinline__ void group_sync(unsigned mask = 0xffffffffu) {
    if constexpr (WARP) __syncwarp(mask);
    else __syncthreads();
}

// Extend-add of all of a front's children (their update blocks' lower triangles) into F,
// with the loads of several children in flight at once.  Each thread queues up to Q entries
// (child k, round m: round m of a child covers its lower-triangle entries tid + m·nt),
// loading every entry's value and its target offset together; then it adds them child by
// child in the children's order with a group barrier between two children (their targets
// may coincide).  Every entry of F thus receives its contributions in the children's order,
// as with one child at a time, and the loads of up to Q rounds cost one round trip.
// ci_of(k) returns the k-th child's record and is called uniformly by the whole group.
template <bool WARP, int Q, class Real, class CI>
__device__ __forceinline__ void extend_add_children(Real* F, int f, const FactorView& a, int nch, const CI& ci_of,
                                                    int tid, int nt, unsigned gmask = 0xffffffffu) {
    int ck = 0, cm = 0;  // cursor: child, round
    while (ck < nch) {
        int qk[Q], off[Q];
        double val[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            qk[q] = -1;
            off[q] = -1;
            val[q] = 0.0;
            if (ck < nch) {
                const ChildInfo ci = ci_of(ck);
                const int r = ci.r, T = r * (r + 1) / 2;
                const int t = tid + cm * nt;
                qk[q] = ck;
                if (t < T) {
                    int i, j;
                    tri_index(t, r, i, j);
                    const int* rel = a.rel + ci.rel_off;
                    off[q] = rel[j] * f + rel[i];
                    val[q] = __ldcg(a.front + ci.u_off + (int64_t)j * ci.fc + i);
                }
                if (++cm * nt >= T) {
                    cm = 0;
                    ++ck;
                }
            }
        }
        int cur = qk[0];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (qk[q] < 0) break;
            if (qk[q] != cur) {
                group_sync<WARP>(gmask);
                cur = qk[q];
            }
            if (off[q] >= 0) F[off[q]] += (Real)val[q];
        }
        group_sync<WARP>(gmask);
    }
}

// The same for a forward solve's gathered vector: v[rel_i] += u_i over the children's
// update vectors (r_k entries each), child by child, several children's loads in flight.
template <int Q, class CI>
__device__ __forceinline__ void gather_children_upd(double* v, const FactorView& a, int nch, const CI& ci_of, int lane) {
    int ck = 0, cm = 0;
    while (ck < nch) {
        int qk[Q], idx[Q];
        double val[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            qk[q] = -1;
            idx[q] = -1;
            val[q] = 0.0;
            if (ck < nch) {
                const ChildInfo ci = ci_of(ck);
                const int i = lane + 32 * cm;
                qk[q] = ck;
                if (i < ci.r) {
                    idx[q] = a.rel[ci.rel_off + i];
                    val[q] = __ldcg(a.upd + ci.rel_off + i);
                }
                if (32 * ++cm >= ci.r) {
                    cm = 0;
                    ++ck;
                }
            }
        }
        int cur = qk[0];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (qk[q] < 0) break;
            if (qk[q] != cur) {
                __syncwarp();
                cur = qk[q];
            }
            if (idx[q] >= 0) v[idx[q]] += val[q];
        }
        __syncwarp();
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
// its serial pivot chain.  Within a panel the columns stay unscaled and thread t owns rows
// k+1+t (+nt …).  One thread computes the pivots: in a warp, thread 0 (it owns row k+1 and,
// as soon as it has applied column k to its own diagonal entry, computes the next pivot and
// its reciprocal while the other lanes apply column k to their rows); in a CTA, the last
// thread, which owns no row of a front of order ≤ nt − 31 and so runs the pivot chain
// (next diagonal entry, pivot, reciprocal) in its own warp, beside the row updates of the
// others: one barrier per column either way.  At the end of the panel the columns are
// scaled in place (L) and their unscaled copy kept in W; then the trailing rank-kPanel
// update gives each thread four independent entries per step, and in a CTA the pivot
// thread first updates the next panel's first diagonal entry and computes its pivot.
// Every entry sees the same operations in the same order whichever thread computes it.
// The pivot signs into bc[kPanel+1 ..] (called by the front's group before its dependency
// wait, so that the global loads are off the critical path; blocked_ldlt's first barrier
// publishes them).
template <class Real>
__device__ __forceinline__ void stage_pivot_signs(Real* bc, int c, int first, const FactorView& a, int tid, int nt) {
    Real* sgn = bc + kPanel + 1;
    for (int k = tid; k < c; k += nt) sgn[k] = a.dsign[first + k] > 0 ? Real(1) : Real(-1);
}

template <bool WARP, class Real = double>
__device__ __forceinline__ int blocked_ldlt(Real* F, Real* W, Real* bc, int f, int c, int first,
                                            const FactorView& a, int tid, int nt, unsigned gmask = 0xffffffffu) {
    int nreg = 0;
    double* dinv = a.dinv + first;
    Real* sgn = bc + kPanel + 1;
    const int piv = WARP ? 0 : nt - 1;  // the thread that computes the pivots
    group_sync<WARP>(gmask);
    auto do_pivot = [&](int k) {  // the pivot thread only
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
    if (tid == piv && c > 0) do_pivot(0);
    for (int k0 = 0; k0 < c; k0 += kPanel) {
        const int nb = min(kPanel, c - k0);
        for (int p = 0; p < nb; ++p) {
            const int k = k0 + p;
            group_sync<WARP>(gmask);  // pivot k and column k final
            const Real* colk = F + (size_t)k * f;
            const Real inv = bc[k % kPanel];
            const int jend = k0 + nb;  // later columns of this panel: k+1 .. jend−1
            if constexpr (!WARP) {
                if (tid == piv && k + 1 < jend) {
                    const Real l = colk[k + 1] * inv;
                    F[(size_t)(k + 1) * f + k + 1] -= l * colk[k + 1];
                    do_pivot(k + 1);
                }
            }
            for (int i = k + 1 + tid; i < f; i += nt) {
                const Real l = colk[i] * inv;
                // in a CTA the diagonal entry (k+1, k+1) belongs to the pivot thread
                const int j0 = (!WARP && i == k + 1) ? k + 2 : k + 1;
                for (int j = j0; j < jend && j <= i; ++j) F[(size_t)j * f + i] -= l * colk[j];
                if (WARP && i == k + 1 && k + 1 < jend) do_pivot(k + 1);  // i == k+1 only for tid 0
            }
        }
        group_sync<WARP>(gmask);
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
        group_sync<WARP>(gmask);
        // trailing rank-nb update of rows/columns k0+nb .. f−1, four entries per thread
        const int base = k0 + nb, m = f - base;
        const Real* L0 = F + (size_t)k0 * f;
        auto trailing = [&](int i, int j) {
            const Real* wr = W + j * kPanel;
            Real x = F[(size_t)j * f + i];
            x -= L0[i] * wr[0];
            if (nb > 1) x -= L0[f + i] * wr[1];
            if (nb > 2) x -= L0[2 * f + i] * wr[2];
            if (nb > 3) x -= L0[3 * f + i] * wr[3];
            return x;
        };
        // in a CTA the pivot thread takes the next pivot's diagonal entry first
        const bool early = !WARP && base < c;
        if (early && tid == piv) {
            F[(size_t)base * f + base] = trailing(base, base);
            do_pivot(base);
        }
        if (m > 0) {
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
                for (int u = 0; u < 4; ++u) acc[u] = trailing(base + ii[u], base + jj[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int tu = t + u * nt;
                    if (tu < T && !(early && tu == 0))
                        F[(size_t)(base + jj[u]) * f + base + ii[u]] = acc[u];
                }
            }
        }
        group_sync<WARP>(gmask);
        if (WARP && tid == piv && base < c) do_pivot(base);
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
    // the front's L (below the diagonal) and D⁻¹ in registers, every load issued before the
    // first FMA (one memory round trip instead of one per column); the solve then runs on
    // register copies with unrolled, bounds-checked loops
    const double* L = a.front + a.front_off[s];
    constexpr int T = kThreadFront;
    double Lr[T * (T - 1) / 2], dr[T], vr[T];
#pragma unroll
    for (int k = 0, e = 0; k < T - 1; ++k)
#pragma unroll
        for (int i = k + 1; i < T; ++i, ++e) Lr[e] = (k < c && i < f) ? L[k * f + i] : 0.0;
#pragma unroll
    for (int i = 0; i < T; ++i) {
        dr[i] = i < c ? a.dinv[first + i] : 0.0;
        vr[i] = i < f ? v[i] : 0.0;
    }
#pragma unroll
    for (int k = 0, e = 0; k < T - 1; e += T - 1 - k, ++k) {
        if (k >= c) break;
        const double xk = vr[k];
#pragma unroll
        for (int i = k + 1; i < T; ++i)
            if (i < f) vr[i] -= Lr[e + i - k - 1] * xk;
    }
    double* u = a.upd + a.upd_off[s];
#pragma unroll
    for (int i = 0; i < T; ++i) {
        if (i < c) w[first + i] = vr[i] * dr[i];
        else if (i < f) u[i - c] = vr[i];
    }
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
    // the known values, L and the permutation in registers, every load issued before the
    // first FMA; then the backward substitution on register copies
    const double* L = a.front + a.front_off[s];
    constexpr int T = kThreadFront;
    double Lr[T * (T - 1) / 2], vr[T];
    int pr[T];
#pragma unroll
    for (int i = 0; i < T; ++i) {
        vr[i] = i < c ? __ldcg(w + first + i) : i < f ? __ldcg(xp + R[i]) : 0.0;
        pr[i] = i < c ? a.perm[first + i] : 0;
    }
#pragma unroll
    for (int k = 0, e = 0; k < T - 1; ++k)
#pragma unroll
        for (int i = k + 1; i < T; ++i, ++e) Lr[e] = (k < c && i < f) ? L[k * f + i] : 0.0;
#pragma unroll
    for (int k = T - 2; k >= 0; --k) {
        if (k < c) {
            const int e = k * (T - 1) - k * (k - 1) / 2;  // start of column k in Lr
            double acc = vr[k];
#pragma unroll
            for (int i = k + 1; i < T; ++i)
                if (i < f) acc -= Lr[e + i - k - 1] * vr[i];
            vr[k] = acc;
        }
    }
#pragma unroll
    for (int i = 0; i < T; ++i) {
        if (i < c) {
            xp[first + i] = vr[i];
            if (accumulate) x[pr[i]] += vr[i];
            else x[pr[i]] = vr[i];
        }
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
// GW: the lanes that work on the front — the whole warp (32), or one half of it (16), when
// a warp holds two fronts of order ≤ kPairFront (their instructions then issue together
// wherever the two fronts' loops agree, which shares the FP64 issue slots, one warp
// instruction occupying a sub-partition's FP64 unit for 64 cycles on this part).  lane is
// the lane in the warp; the group's lanes are lane & ~(GW−1) … + GW−1.  wait() is called
// by the group alone.
template <class Wait, class Real = double, int EAQ = 8, int GW = 32>
__device__ __forceinline__ bool warp_factor_front(int s, const FactorView& a, const double* __restrict__ kval,
                                                  Real* F, Real* lk, int lane, const Wait& wait) {
    static_assert(GW == 32 || GW == 16, "a front takes a warp or half of one");
    const unsigned gmask = GW == 32 ? 0xffffffffu : (0xffffu << (lane & 16));
    const int gl = lane & (GW - 1);  // lane in the group
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    const int ff = f * f;
    for (int i = gl; i < ff; i += GW) F[i] = Real(0);
    __syncwarp(gmask);
    // original entries (static regularisation on the diagonal): loads first, then stores
    {
        const int64_t e0 = a.amap_ptr[s], e1 = a.amap_ptr[s + 1];
        for (int64_t e = e0 + gl; e < e1; e += 4 * GW) {
            int off[4];
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t eu = e + u * GW;
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
    // child records of the first GW children, one per lane, and the pivot signs (loaded
    // before the wait)
    const int k0 = a.child_ptr[s], nch = a.child_ptr[s + 1] - k0;
    ChildInfo mine;
    if (gl < nch) mine = a.cinfo[k0 + gl];
    stage_pivot_signs(lk + kPanel * f, c, first, a, gl, GW);
    __syncwarp(gmask);
    if (!wait()) return false;
    // extend-add of the children's update blocks, several children's loads in flight
    auto ci_of = [&](int k) {
        ChildInfo ci;
        if (k < GW) {
            ci.u_off = __shfl_sync(gmask, mine.u_off, k, GW);
            ci.rel_off = __shfl_sync(gmask, mine.rel_off, k, GW);
            ci.fc = __shfl_sync(gmask, mine.fc, k, GW);
            ci.r = __shfl_sync(gmask, mine.r, k, GW);
        } else {
            ci = a.cinfo[k0 + k];
        }
        return ci;
    };
    extend_add_children<true, EAQ, Real>(F, f, a, nch, ci_of, gl, GW, gmask);
    const int nreg = blocked_ldlt<true, Real>(F, lk, lk + kPanel * f, f, c, first, a, gl, GW, gmask);
    double* G = a.front + a.front_off[s];
    for (int i = gl; i < ff; i += GW) G[i] = (double)F[i];
    if (gl == 0 && nreg) atomicAdd(a.nreg, nreg);
    __syncwarp(gmask);
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

// LOADP = false: P already holds the panel (the front just factored, leading dimension f)
template <class Wait, int EAQ = 8, bool LOADP = true>
__device__ __forceinline__ bool warp_fwd_front(int s, const FactorView& a, const double* __restrict__ rhs,
                                               double* __restrict__ w, double* v, const double* P, int lane,
                                               const Wait& wait) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    if (LOADP) warp_load_panel(a.front + a.front_off[s], f * c, const_cast<double*>(P), lane);
    for (int i = lane; i < f; i += 32) v[i] = i < c ? rhs[a.perm[first + i]] : 0.0;
    const int k0 = a.child_ptr[s], nch = a.child_ptr[s + 1] - k0;
    ChildInfo mine;
    if (lane < nch) mine = a.cinfo[k0 + lane];
    // the pivot reciprocals of the front's columns (c ≤ 64), loaded before the wait
    const double* dinv = a.dinv + first;
    const double dv0 = lane < c ? dinv[lane] : 0.0, dv1 = lane + 32 < c ? dinv[lane + 32] : 0.0;
    __syncwarp();
    if (!wait()) return false;
    auto ci_of = [&](int k) {
        ChildInfo ci{0, 0, 0, 0};
        if (k < 32) {
            ci.rel_off = __shfl_sync(0xffffffffu, mine.rel_off, k);
            ci.r = __shfl_sync(0xffffffffu, mine.r, k);
        } else {
            ci = a.cinfo[k0 + k];
        }
        return ci;
    };
    gather_children_upd<EAQ>(v, a, nch, ci_of, lane);
    for (int k = 0; k < c; ++k) {
        const double xk = v[k];
        const double* colk = P + k * f;
        for (int i = k + 1 + lane; i < f; i += 32) v[i] -= colk[i] * xk;
        __syncwarp();
    }
    if (lane < c) w[first + lane] = v[lane] * dv0;
    if (lane + 32 < c) w[first + lane + 32] = v[lane + 32] * dv1;
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
    const int p0 = lane < c ? a.perm[first + lane] : 0, p1 = lane + 32 < c ? a.perm[first + lane + 32] : 0;
    if (!wait()) return false;
    if (lane < f) v[lane] = __ldcg(lane < c ? w + first + lane : xp + r0);
    if (lane + 32 < f) v[lane + 32] = __ldcg(lane + 32 < c ? w + first + lane + 32 : xp + r1);
    __syncwarp();
    // the solved entries below the pivot block (i ≥ c) into each pivot row k < c: a register
    // sum per lane in two interleaved partial sums (v_i for i ≥ c is read-only here, so the
    // FMAs of one lane do not wait on shared memory)
    for (int k = lane; k < c; k += 32) {
        double a0 = v[k], a1 = 0.0;
        int i = c;
        for (; i + 1 < f; i += 2) {
            a0 -= P[k * f + i] * v[i];
            a1 -= P[k * f + i + 1] * v[i + 1];
        }
        if (i < f) a0 -= P[k * f + i] * v[i];
        v[k] = a0 + a1;
    }
    __syncwarp();
    for (int i = c - 1; i > 0; --i) {
        const double xi = v[i];
        for (int k = lane; k < i; k += 32) v[k] -= P[k * f + i] * xi;
        __syncwarp();
    }
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i >= c) break;
        const double xi = v[i];
        const int pi = h ? p1 : p0;
        xp[first + i] = xi;
        if (accumulate) x[pi] += xi;
        else x[pi] = xi;
    }
    __syncwarp();
    return true;
}

}  // namespace qoco
