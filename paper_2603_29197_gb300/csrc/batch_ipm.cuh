// Device code of the persistent batched kernel (instantiated in batch_ipm_f64.cu and
// batch_ipm_mixed.cu).  Batched problems in one persistent launch: every CTA takes whole instances of eq. (1)
// from a queue (largest first) and runs the complete predictor–corrector interior-point
// method of each on chip — initial point, then per iteration the residuals and stopping
// test, NT scaling and −W² (paper §2.1), the LDLᵀ factorisation of the instance's block
// of the KKT matrix of eq. (2) and its two solves with refinement (§2.2), steps and
// update — with block barriers between the steps and no wait on any other CTA.  The
// arithmetic is that of the single-problem kernels (the same front, cone and Jordan
// algebra device functions), per instance: residual norms, gap, μ, σ, the step lengths,
// the refinement's backward error (‖r − Kx‖∞ / (‖K‖∞‖x‖∞ + ‖r‖∞) over the instance's rows)
// and the stopping test all belong to one instance, as in a one-problem solve.
#pragma once

#include "batch_ipm.h"
#include "cones.cuh"
#include "fronts.cuh"

namespace qoco {
namespace batch_ipm_detail {
namespace {  // internal linkage: each translation unit instantiating the kernel has its own copy

// Rows of one instance in the stacked system: x rows, y rows, orthant z rows and SOC z
// rows, each a contiguous range of the stack; the cone entries (s, z, W data) of the
// instance are the orthant range [o0, o1) and the SOC range [q0, q1) of the m-vector.
struct Rows {
    int n, p;               // stacked x and y dimensions
    int x0, nx, y0, ny, o0, no, q0, nq;
    int k0, k1;             // the instance's SOCs
    int total;
    __device__ void init(const BatchIPMArgs& A, int i) {
        const BatchView& B = A.B;
        n = A.K.n;
        p = A.K.p;
        x0 = B.xo[i]; nx = B.xo[i + 1] - x0;
        y0 = B.yo[i]; ny = B.yo[i + 1] - y0;
        o0 = B.lo[i]; no = B.lo[i + 1] - o0;
        q0 = A.L + B.so[i]; nq = A.L + B.so[i + 1] - q0;
        k0 = B.ko[i]; k1 = B.ko[i + 1];
        total = nx + ny + no + nq;
    }
    // k-th row of the instance (0 ≤ k < total) as a KKT row index
    __device__ __forceinline__ int row(int k) const {
        if (k < nx) return x0 + k;
        k -= nx;
        if (k < ny) return n + y0 + k;
        k -= ny;
        if (k < no) return n + p + o0 + k;
        return n + p + q0 + (k - no);
    }
};

__device__ __forceinline__ double bits_max(double a, double b) {  // non-negative, NaN on top
    return __double_as_longlong(b) > __double_as_longlong(a) ? b : a;
}
__device__ __forceinline__ double bits_min(double a, double b) {  // non-negative or +inf
    return __double_as_longlong(b) < __double_as_longlong(a) ? b : a;
}

// Block reduction of NV values (sums, or maxima / minima of non-negative values through
// their bit patterns); every thread returns the totals, combined in a fixed order.
// kind[k]: 0 sum, 1 max, 2 min.  sm: NV·(warps per block) doubles.
template <int NV>
__device__ void cta_reduce(double (&v)[NV], const int (&kind)[NV], double* sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double a = v[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double b = __shfl_xor_sync(0xffffffffu, a, o);
            a = kind[k] == 0 ? a + b : kind[k] == 1 ? bits_max(a, b) : bits_min(a, b);
        }
        if (lane == 0) sm[k * nw + wid] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double a = sm[k * nw];
        for (int w = 1; w < nw; ++w) {
            const double b = sm[k * nw + w];
            a = kind[k] == 0 ? a + b : kind[k] == 1 ? bits_max(a, b) : bits_min(a, b);
        }
        v[k] = a;
    }
    __syncthreads();
}

__device__ __forceinline__ int take(unsigned int* next) {
    __shared__ int s_i;
    if (threadIdx.x == 0) s_i = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int i = s_i;
    __syncthreads();
    return i;
}

// ---- factorisation and solves of the instance's tree (level by level) ----------------
// Real: the fronts' working type (FP64, or FP32 in mixed precision: L and D are stored in
// FP64 either way and the solves and refinement run in FP64)
template <int NW, class Real>
__device__ __noinline__ void inst_factor(const BatchIPMArgs& A, int inst, double* F) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Real* Fr = reinterpret_cast<Real*>(F);
    for (int k = A.lv_ptr[inst]; k < A.lv_ptr[inst + 1]; ++k) {
        const int t0 = A.ent[3 * k], w0 = A.ent[3 * k + 1], e1 = A.ent[3 * k + 2];
        for (int t = t0 + (int)threadIdx.x; t < w0; t += NW * 32)
            thread_factor_front<NoWait, Real>(A.sched[t], A.F, A.kval, NoWait());
        for (int t = w0 + wid; t < e1; t += NW)
            warp_factor_front<NoWait, Real, 4>(A.sched[t], A.F, A.kval, Fr, Fr + A.fmax * A.fmax, lane, NoWait());
        __syncthreads();
    }
}

// x = (LDLᵀ)⁻¹ rhs on the instance's entries (x[perm] written, or added when acc)
template <int NW>
__device__ __noinline__ void inst_solve(const BatchIPMArgs& A, int inst, const double* rhs, double* x, int acc, double* V) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* P = V + A.fmax;
    const int k0 = A.lv_ptr[inst], k1 = A.lv_ptr[inst + 1];
    for (int k = k0; k < k1; ++k) {
        const int t0 = A.ent[3 * k], w0 = A.ent[3 * k + 1], e1 = A.ent[3 * k + 2];
        for (int t = t0 + (int)threadIdx.x; t < w0; t += NW * 32) thread_fwd_front(A.sched[t], A.F, rhs, A.sol_w, NoWait());
        for (int t = w0 + wid; t < e1; t += NW) warp_fwd_front<NoWait, 4>(A.sched[t], A.F, rhs, A.sol_w, V, P, lane, NoWait());
        __syncthreads();
    }
    for (int k = k1 - 1; k >= k0; --k) {
        const int t0 = A.ent[3 * k], w0 = A.ent[3 * k + 1], e1 = A.ent[3 * k + 2];
        for (int t = t0 + (int)threadIdx.x; t < w0; t += NW * 32)
            thread_bwd_front(A.sched[t], A.F, A.sol_w, A.sol_xp, x, acc, NoWait());
        for (int t = w0 + wid; t < e1; t += NW)
            warp_bwd_front(A.sched[t], A.F, A.sol_w, A.sol_xp, x, acc, V, P, lane, NoWait());
        __syncthreads();
    }
}

// ‖K‖∞ over the instance's rows (the refinement's scale)
__device__ __noinline__ double inst_normK(const BatchIPMArgs& A, const Rows& R, double* red) {
    double v[1] = {0.0};
    for (int k = threadIdx.x; k < R.total; k += blockDim.x) {
        const int row = R.row(k);
        double a = 0.0;
        for (int64_t t = A.K.rowptr[row]; t < A.K.rowptr[row + 1]; ++t) a += fabs(A.kval[t]);
        v[0] = bits_max(v[0], a);
    }
    const int kind[1] = {1};
    cta_reduce<1>(v, kind, red);
    return v[0];
}

// res = r − K x on the instance's rows; returns the backward error (NaN when a value is
// not finite)
// cw (optional): the componentwise backward error, computed only when asked for
__device__ __noinline__ double inst_residual(const BatchIPMArgs& A, const Rows& R, const double* x, const double* r,
                                double* res, double normK, double* red, double* cw) {
    // ‖res‖∞, ‖x‖∞, ‖r‖∞, max_i |res_i| / (|K||x| + |r|)_i (componentwise)
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const bool want_cw = cw != nullptr;
    for (int k = threadIdx.x; k < R.total; k += blockDim.x) {
        const int row = R.row(k);
        double a = r[row], d = fabs(r[row]);
        for (int64_t t = A.K.rowptr[row]; t < A.K.rowptr[row + 1]; ++t) {
            const double kx = A.kval[t] * x[A.K.colidx[t]];
            a -= kx;
            if (want_cw) d += fabs(kx);
        }
        res[row] = a;
        v[0] = amax(v[0], a);
        v[1] = amax(v[1], x[row]);
        v[2] = amax(v[2], r[row]);
        if (want_cw)
            v[3] = amax(v[3], d > 0.0 ? a / d : (a == 0.0 ? 0.0 : a * __longlong_as_double(0x7ff0000000000000LL)));
    }
    const int kind[4] = {1, 1, 1, 1};
    cta_reduce<4>(v, kind, red);
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2])) {
        if (want_cw) *cw = nan;
        return nan;
    }
    if (want_cw) *cw = v[3];
    const double den = normK * v[1] + v[2];
    return den > 0.0 ? v[0] / den : 0.0;
}

// x = K_ε⁻¹ r refined against K to the backward-error target (≤ max_refine steps);
// returns whether the target was reached.  cw: the componentwise backward error must
// reach it too (solves on an FP32 factor: near the end of a solve ‖K‖∞ is ~1e16, and a
// solve that met the normwise target alone could still be wrong in the rows of small
// scale, which slowed or broke the instance's iteration)
template <int NW>
__device__ bool inst_solve_refine(const BatchIPMArgs& A, int inst, const Rows& R, const double* r, double* x,
                                  double normK, double* V, double* red, bool cw) {
    inst_solve<NW>(A, inst, r, x, 0, V);
    for (int steps = 0;; ++steps) {
        double bcw = 0.0;
        const double be = inst_residual(A, R, x, r, A.res, normK, red, cw ? &bcw : nullptr);
        if (be <= A.refine_tol && (!cw || bcw <= A.refine_tol)) return true;
        if (!(be == be) || steps >= A.max_refine) return false;  // NaN, or out of steps
        inst_solve<NW>(A, inst, A.res, x, 1, V);
    }
}

// One solve of the iteration with the current factor; in mixed precision a solve whose
// refinement misses its target on an FP32 factor refactors the instance in FP64 and
// solves again (fp32 then says whether the current factor is FP32).
template <int NW, bool MIX>
__device__ void inst_solve_mixed(const BatchIPMArgs& A, int inst, const Rows& R, const double* r, double* x,
                                 double normK, double* V, double* red, bool& fp32, int& fails) {
    const bool ok = inst_solve_refine<NW>(A, inst, R, r, x, normK, V, red, MIX && fp32);
    if (MIX && fp32) {
        if (ok) { fails = 0; return; }
        ++fails;
        fp32 = false;
        inst_factor<NW, double>(A, inst, V);
        inst_solve_refine<NW>(A, inst, R, r, x, normK, V, red, false);
    }
}

// ---- cone operations over the instance's cones (orthant: one thread per entry; SOC of
// dimension ≤ kSmallCone: one thread; larger: one warp) -------------------------------
template <class FO, class FS1, class FS32>
__device__ __forceinline__ void for_cones(const BatchIPMArgs& A, const Rows& R, FO fo, FS1 fs1, FS32 fs32) {
    for (int i = R.o0 + (int)threadIdx.x; i < R.o0 + R.no; i += blockDim.x) fo(i);
    for (int k = R.k0 + (int)threadIdx.x; k < R.k1; k += blockDim.x)
        if (A.C.dim[k] <= kSmallCone) fs1(k, A.C.off[k], A.C.dim[k]);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = R.k0 + wid; k < R.k1; k += nw)
        if (A.C.dim[k] > kSmallCone) fs32(k, A.C.off[k], A.C.dim[k], lane);
    __syncthreads();
}

// largest step keeping u1 + α du1 and u2 + α du2 in the instance's cone
__device__ __noinline__ double inst_max_step(const BatchIPMArgs& A, const Rows& R, const double* u1, const double* du1,
                                const double* u2, const double* du2, double* red) {
    double v[1] = {INFINITY};
    for (int i = R.o0 + (int)threadIdx.x; i < R.o0 + R.no; i += blockDim.x) {
        if (du1[i] < 0.0) v[0] = fmin(v[0], -u1[i] / du1[i]);
        if (du2[i] < 0.0) v[0] = fmin(v[0], -u2[i] / du2[i]);
    }
    for (int k = R.k0 + (int)threadIdx.x; k < R.k1; k += blockDim.x) {
        const int o = A.C.off[k], d = A.C.dim[k];
        if (d <= kSmallCone) v[0] = fmin(v[0], fmin(soc_step<1>(o, d, 0, u1, du1), soc_step<1>(o, d, 0, u2, du2)));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = R.k0 + wid; k < R.k1; k += nw) {
        const int o = A.C.off[k], d = A.C.dim[k];
        if (d > kSmallCone) {
            const double a = fmin(soc_step<32>(o, d, lane, u1, du1), soc_step<32>(o, d, lane, u2, du2));
            v[0] = fmin(v[0], a);
        }
    }
    const int kind[1] = {2};
    cta_reduce<1>(v, kind, red);
    return v[0];
}

// the initial point's shift measure of u: max over cones of −u_i (orthant) and ‖u_1‖ − u_0
__device__ __noinline__ double inst_shift_measure(const BatchIPMArgs& A, const Rows& R, const double* u, double* red) {
    double v[1] = {-INFINITY};
    for (int i = R.o0 + (int)threadIdx.x; i < R.o0 + R.no; i += blockDim.x) v[0] = fmax(v[0], -u[i]);
    for (int k = R.k0 + (int)threadIdx.x; k < R.k1; k += blockDim.x) {
        const int o = A.C.off[k], d = A.C.dim[k];
        double a = 0.0;
        for (int j = 1; j < d; ++j) a += u[o + j] * u[o + j];
        v[0] = fmax(v[0], sqrt(a) - u[o]);
    }
    // max through −min of the negated values (fixed-order block reduction)
    __shared__ double sm[32];
    double a = v[0];
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    a = sm[0];
    for (int w = 1; w < nw; ++w) a = fmax(a, sm[w]);
    __syncthreads();
    (void)red;
    return a;
}

// right-hand side of the z rows for d_s (see k_rhs_z), on the instance's cones
__device__ __noinline__ void inst_rhs_z(const BatchIPMArgs& A, const Rows& R, const double* rz, const double* dsa,
                           const double* dza, double smu, bool combined, double* rhs_z) {
    for_cones(
        A, R,
        [&](int i) {
            const double li = A.lam[i], wi = A.wbar[i];
            double ds = -li * li;
            if (combined) ds += -(dsa[i] / wi) * (wi * dza[i]) + smu;
            const double ti = ds / li;
            A.t[i] = ti;
            rhs_z[i] = -rz[i] - wi * ti;
        },
        [&](int k, int o, int d) {
            soc_rhs<1>(k, o, d, 0, A.C, A.lam, A.wbar, A.eta, rz, dsa, dza, smu, combined, A.t, A.t1, A.t2, rhs_z);
        },
        [&](int k, int o, int d, int lane) {
            soc_rhs<32>(k, o, d, lane, A.C, A.lam, A.wbar, A.eta, rz, dsa, dza, smu, combined, A.t, A.t1, A.t2,
                        rhs_z);
        });
}

// W = I in the instance's −W² slots (the initial point)
__device__ __noinline__ void inst_w2_identity(const BatchIPMArgs& A, const Rows& R) {
    for_cones(
        A, R, [&](int i) { A.kval[A.w2slot[i]] = -1.0; },
        [&](int k, int o, int d) {
            const int64_t* sl = A.w2slot + A.L + A.w2ptr[k];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) A.kval[sl[(int64_t)a * d + b]] = a == b ? -1.0 : 0.0;
        },
        [&](int k, int o, int d, int lane) {
            const int64_t* sl = A.w2slot + A.L + A.w2ptr[k];
            for (int64_t e = lane; e < (int64_t)d * d; e += 32) {
                const int a = (int)(e / d), b = (int)(e - (int64_t)a * d);
                A.kval[sl[e]] = a == b ? -1.0 : 0.0;
            }
        });
}

// NT scaling of the instance's cones and −W² into its KKT value slots
__device__ __noinline__ void inst_nt_scaling(const BatchIPMArgs& A, const Rows& R, const double* z) {
    for_cones(
        A, R,
        [&](int i) {
            const double si = A.s[i], zi = z[i];
            A.wbar[i] = sqrt(si / zi);
            A.lam[i] = sqrt(si * zi);
            A.kval[A.w2slot[i]] = -(si / zi);
        },
        [&](int k, int o, int d) {
            soc_nt<1>(k, o, d, 0, A.s, z, A.wbar, A.eta, A.lam, A.kval, A.w2slot + A.L + A.w2ptr[k]);
        },
        [&](int k, int o, int d, int lane) {
            soc_nt<32>(k, o, d, lane, A.s, z, A.wbar, A.eta, A.lam, A.kval, A.w2slot + A.L + A.w2ptr[k]);
        });
}

// Δs = W(t − WΔz)
__device__ __noinline__ void inst_ds(const BatchIPMArgs& A, const Rows& R, const double* dz, double* ds) {
    for_cones(
        A, R,
        [&](int i) {
            const double wi = A.wbar[i];
            ds[i] = wi * (A.t[i] - wi * dz[i]);
        },
        [&](int k, int o, int d) {
            soc_W<1>(o, d, 0, A.wbar, A.eta[k], dz, A.t1, false);
            for (int a = 0; a < d; ++a) A.t1[o + a] = A.t[o + a] - A.t1[o + a];
            soc_W<1>(o, d, 0, A.wbar, A.eta[k], A.t1, ds, false);
        },
        [&](int k, int o, int d, int lane) {
            soc_W<32>(o, d, lane, A.wbar, A.eta[k], dz, A.t1, false);
            __syncwarp();
            for (int a = lane; a < d; a += 32) A.t1[o + a] = A.t[o + a] - A.t1[o + a];
            __syncwarp();
            soc_W<32>(o, d, lane, A.wbar, A.eta[k], A.t1, ds, false);
        });
}

// r = [Px + c + Aᵀy + Gᵀz; Ax − b; Gx + s − h] on the instance's rows and the quantities
// of its stopping test: sums xᵀPx, cᵀx, bᵀy, hᵀz, sᵀz; maxima ‖Px‖∞, ‖Aᵀy‖∞, ‖Gᵀz‖∞, ‖Ax‖∞,
// ‖Gx‖∞, ‖r_x‖∞, ‖r_y‖∞, ‖r_z‖∞, ‖s‖∞ (in that order in v)
__device__ __noinline__ void inst_stop_quantities(const BatchIPMArgs& A, const Rows& R, double (&v)[14],
                                                  double* red) {
    const int n = R.n, np = R.n + R.p;
    for (int k = 0; k < 14; ++k) v[k] = 0.0;
    for (int k = threadIdx.x; k < R.total; k += blockDim.x) {
        const int row = R.row(k);
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int64_t t = A.K.rowptr[row]; t < A.K.rowptr[row + 1]; ++t) {
            const int j = A.K.colidx[t];
            const double kv = A.kval[t] * A.xyz[j];
            if (j < n) a0 += kv;
            else if (j < np) a1 += kv;
            else a2 += kv;
        }
        if (row < n) {
            const double x = A.xyz[row], rv = a0 + A.c[row] + a1 + a2;
            A.r[row] = rv;
            v[0] += x * a0;
            v[1] += A.c[row] * x;
            v[5] = amax(v[5], a0);
            v[6] = amax(v[6], a1);
            v[7] = amax(v[7], a2);
            v[10] = amax(v[10], rv);
        } else if (row < np) {
            const double rv = a0 - A.b[row - n];
            A.r[row] = rv;
            v[2] += A.b[row - n] * A.xyz[row];
            v[8] = amax(v[8], a0);
            v[11] = amax(v[11], rv);
        } else {
            const int i = row - np;
            const double rv = a0 + A.s[i] - A.h[i];
            A.r[row] = rv;
            v[3] += A.h[i] * A.xyz[row];
            v[4] += A.s[i] * A.xyz[row];
            v[9] = amax(v[9], a0);
            v[12] = amax(v[12], rv);
            v[13] = amax(v[13], A.s[i]);
        }
    }
    const int kind[14] = {0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1};
    cta_reduce<14>(v, kind, red);
}

template <int NW, bool MIX>
__device__ void solve_instance(const BatchIPMArgs& A, int inst, double* Fw, double* red) {
    const BatchView& B = A.B;
    Rows R;
    R.init(A, inst);
    const int n = R.n, p = R.p, np = n + p;
    double* z = A.xyz + np;
    // ---- initial point: W = I, [x; y; z] = K_ε⁻¹[−c; b; h], s = −z, shift into the cone
    inst_w2_identity(A, R);
    // mixed precision: FP32 fronts unless the instance's last two FP32 factors failed
    int fails = 0;
    bool fp32 = MIX;
    if (fp32) inst_factor<NW, float>(A, inst, Fw);
    else inst_factor<NW, double>(A, inst, Fw);
    double normK = inst_normK(A, R, red);
    for (int k = threadIdx.x; k < R.total; k += blockDim.x) {
        const int row = R.row(k);
        A.rhs[row] = row < n ? -A.c[row] : row < np ? A.b[row - n] : A.h[row - np];
    }
    __syncthreads();
    inst_solve_mixed<NW, MIX>(A, inst, R, A.rhs, A.d_cmb, normK, Fw, red, fp32, fails);
    for (int k = threadIdx.x; k < R.total; k += blockDim.x) {
        const int row = R.row(k);
        A.xyz[row] = A.d_cmb[row];
        if (row >= np) A.s[row - np] = -A.d_cmb[row];
    }
    __syncthreads();
    const double ms = inst_shift_measure(A, R, A.s, red);
    const double mz = inst_shift_measure(A, R, z, red);
    for_cones(
        A, R,
        [&](int i) {
            if (ms >= 0.0) A.s[i] += 1.0 + ms;
            if (mz >= 0.0) z[i] += 1.0 + mz;
        },
        [&](int k, int o, int d) {
            if (ms >= 0.0) A.s[o] += 1.0 + ms;
            if (mz >= 0.0) z[o] += 1.0 + mz;
        },
        [&](int k, int o, int d, int lane) {
            if (lane == 0 && ms >= 0.0) A.s[o] += 1.0 + ms;
            if (lane == 0 && mz >= 0.0) z[o] += 1.0 + mz;
        });

    const double nu = B.nu[inst];
    int conv = 0, conv_inacc = 0, nonfinite = 0, it_done = A.max_iter;
    for (int it = 0;; ++it) {
        // ---- residuals and the stopping test (the norms and max-sets of one problem)
        double v[14];
        inst_stop_quantities(A, R, v, red);
        const double pobj = 0.5 * v[0] + v[1], dobj = -0.5 * v[0] - v[2] - v[3], gap = v[4];
        const double mu = nu > 0.0 ? gap / nu : 0.0;
        bool finite = isfinite(pobj) && isfinite(dobj) && isfinite(gap);
        for (int k = 5; k < 14; ++k) finite = finite && isfinite(v[k]);
        auto test = [&](double ea, double er) {
            const bool oy = v[11] <= ea + er * fmax(v[8], B.b_inf[inst]);
            const bool oz = v[12] <= ea + er * fmax(v[9], fmax(v[13], B.h_inf[inst]));
            const bool ox = v[10] <= ea + er * fmax(fmax(v[5], v[6]), fmax(v[7], B.c_inf[inst]));
            const bool og = fabs(gap) <= ea + er * fmax(1.0, fmax(fabs(pobj), fabs(dobj)));
            return ox && oy && oz && og;
        };
        if (threadIdx.x == 0) {
            B.pobj[inst] = pobj;
            B.dobj[inst] = dobj;
            B.gap[inst] = gap;
            B.mu[inst] = mu;
            B.res[3 * inst] = v[10];
            B.res[3 * inst + 1] = v[11];
            B.res[3 * inst + 2] = v[12];
        }
        if (!finite) { nonfinite = 1; it_done = it; break; }
        if (test(A.abstol, A.reltol)) { conv = 1; it_done = it; break; }
        if (it >= A.max_iter) { conv_inacc = test(A.abstol_inacc, A.reltol_inacc) ? 1 : 0; break; }

        // ---- NT scaling, −W² into the KKT values, factorisation
        inst_nt_scaling(A, R, z);
        fp32 = MIX && fails < 2;
        if (fp32) inst_factor<NW, float>(A, inst, Fw);
        else inst_factor<NW, double>(A, inst, Fw);
        normK = inst_normK(A, R, red);
        // ---- predictor
        for (int k = threadIdx.x; k < R.nx + R.ny; k += blockDim.x) {
            const int row = R.row(k);
            A.rhs[row] = -A.r[row];
        }
        inst_rhs_z(A, R, A.r + np, nullptr, nullptr, 0.0, false, A.rhs + np);
        inst_solve_mixed<NW, MIX>(A, inst, R, A.rhs, A.d_aff, normK, Fw, red, fp32, fails);
        inst_ds(A, R, A.d_aff + np, A.ds_aff);
        const double aa = fmin(1.0, inst_max_step(A, R, A.s, A.ds_aff, z, A.d_aff + np, red));
        const double smu = pow(1.0 - aa, 3.0) * mu;
        // ---- corrector
        for (int k = threadIdx.x; k < R.nx + R.ny; k += blockDim.x) {
            const int row = R.row(k);
            A.rhs[row] = -A.r[row];
        }
        inst_rhs_z(A, R, A.r + np, A.ds_aff, A.d_aff + np, smu, true, A.rhs + np);
        inst_solve_mixed<NW, MIX>(A, inst, R, A.rhs, A.d_cmb, normK, Fw, red, fp32, fails);
        inst_ds(A, R, A.d_cmb + np, A.ds_cmb);
        const double amx = inst_max_step(A, R, A.s, A.ds_cmb, z, A.d_cmb + np, red);
        const double alpha = fmin(1.0, A.step_fraction * amx);
        for (int k = threadIdx.x; k < R.total; k += blockDim.x) {
            const int row = R.row(k);
            A.xyz[row] += alpha * A.d_cmb[row];
            if (row >= np) A.s[row - np] += alpha * A.ds_cmb[row - np];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        B.conv[inst] = conv;
        B.conv_inacc[inst] = conv || conv_inacc;
        B.nonfinite[inst] = nonfinite;
        B.iters[inst] = it_done;
    }
    __syncthreads();
}

// NW warps per CTA; MINB resident CTAs per SM asked of the compiler (16/NW: up to 128
// registers per thread; 32/NW: 64 registers, twice the instances in flight per SM)
template <int NW, int MINB, bool MIX>
__global__ void __launch_bounds__(NW * 32, MINB) k_batch_ipm(BatchIPMArgs A) {
    extern __shared__ double smem[];
    __shared__ double red[14 * NW];
    double* Fw = smem + (size_t)(threadIdx.x >> 5) * wfactor_stride(A.fmax);
    for (;;) {
        const int q = take(A.next);
        if (q >= A.B.nb) return;
        solve_instance<NW, MIX>(A, A.order[q], Fw, red);
    }
}

}  // namespace
}  // namespace batch_ipm_detail
}  // namespace qoco
