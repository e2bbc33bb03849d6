// Batched problems: many independent instances of eq. (1) solved by one interior-point
// loop over their block-diagonal stack.  The KKT matrix of eq. (2) is then block diagonal
// and its supernodal tree a forest, so the factorisation and the solves need nothing
// new; what changes is that every scalar of the method (paper §2: the residual norms,
// the gap and μ, the step lengths, σ) belongs to one instance.  These kernels compute
// them per instance — one warp per instance over its contiguous row segments, in a fixed
// order, so the sums are deterministic — and apply per-instance steps.  An instance that
// has met the stopping test takes zero steps from then on.
#include <cuda_runtime.h>

#include "batch.h"
#include "cones.cuh"
#include "row_kernels.h"

namespace qoco {

namespace {

// r = [Px + c + Aᵀy + Gᵀz; Ax − b; Gx + s − h] (one thread per KKT row), and the
// per-row products the stopping test scales with: aux[3i..3i+2] = (Px, Aᵀy, Gᵀz) on x
// rows, (Ax, ·, ·) on y rows, (Gx, ·, ·) on z rows
__global__ void k_batch_residual(KKTView K, const double* __restrict__ xyz, const double* __restrict__ s,
                                 const double* __restrict__ c, const double* __restrict__ b,
                                 const double* __restrict__ h, double* __restrict__ r, double* __restrict__ aux) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= K.N) return;
    const int n = K.n, p = K.p;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t t = K.rowptr[row]; t < K.rowptr[row + 1]; ++t) {
        const int j = K.colidx[t];
        const double kv = K.val[t] * xyz[j];
        if (j < n) a0 += kv;
        else if (j < n + p) a1 += kv;
        else a2 += kv;
    }
    double rv;
    if (row < n) rv = a0 + c[row] + a1 + a2;
    else if (row < n + p) rv = a0 - b[row - n];
    else rv = a0 + s[row - n - p] - h[row - n - p];
    r[row] = rv;
    aux[3 * (int64_t)row] = a0;
    aux[3 * (int64_t)row + 1] = a1;
    aux[3 * (int64_t)row + 2] = a2;
}

struct Acc {
    double xPx = 0, cx = 0, by = 0, hz = 0, sz = 0;
    double Px = 0, Aty = 0, Gtz = 0, Ax = 0, Gx = 0, rx = 0, ry = 0, rz = 0, s = 0;
};

__device__ __forceinline__ double wmax(double v) { return warp_max_nonneg(v); }

// one warp per instance: its stopping test (same norms and max-sets as the single
// problem), objective values, gap and μ
__global__ void k_batch_reduce(BatchView B, int n, int p, int L, const double* __restrict__ xyz,
                               const double* __restrict__ s, const double* __restrict__ c,
                               const double* __restrict__ b, const double* __restrict__ h,
                               const double* __restrict__ r, const double* __restrict__ aux, int iter,
                               double abstol, double reltol, double abstol_inacc, double reltol_inacc) {
    const int lane = threadIdx.x & 31;
    const int inst = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (inst >= B.nb) return;
    Acc a;
    for (int i = B.xo[inst] + lane; i < B.xo[inst + 1]; i += 32) {
        const double x = xyz[i], px = aux[3 * (int64_t)i];
        a.xPx += x * px;
        a.cx += c[i] * x;
        a.Px = amax(a.Px, px);
        a.Aty = amax(a.Aty, aux[3 * (int64_t)i + 1]);
        a.Gtz = amax(a.Gtz, aux[3 * (int64_t)i + 2]);
        a.rx = amax(a.rx, r[i]);
    }
    for (int j = B.yo[inst] + lane; j < B.yo[inst + 1]; j += 32) {
        const int row = n + j;
        a.by += b[j] * xyz[row];
        a.Ax = amax(a.Ax, aux[3 * (int64_t)row]);
        a.ry = amax(a.ry, r[row]);
    }
    // z rows: the instance's orthant entries, then its SOC entries
    for (int seg = 0; seg < 2; ++seg) {
        const int lo = seg == 0 ? B.lo[inst] : L + B.so[inst];
        const int hi = seg == 0 ? B.lo[inst + 1] : L + B.so[inst + 1];
        for (int i = lo + lane; i < hi; i += 32) {
            const int row = n + p + i;
            const double zi = xyz[row];
            a.hz += h[i] * zi;
            a.sz += s[i] * zi;
            a.Gx = amax(a.Gx, aux[3 * (int64_t)row]);
            a.rz = amax(a.rz, r[row]);
            a.s = amax(a.s, s[i]);
        }
    }
    a.xPx = warp_sum(a.xPx); a.cx = warp_sum(a.cx); a.by = warp_sum(a.by);
    a.hz = warp_sum(a.hz); a.sz = warp_sum(a.sz);
    a.Px = wmax(a.Px); a.Aty = wmax(a.Aty); a.Gtz = wmax(a.Gtz); a.Ax = wmax(a.Ax);
    a.Gx = wmax(a.Gx); a.rx = wmax(a.rx); a.ry = wmax(a.ry); a.rz = wmax(a.rz); a.s = wmax(a.s);
    if (lane) return;
    const double pobj = 0.5 * a.xPx + a.cx;
    const double dobj = -0.5 * a.xPx - a.by - a.hz;
    const double nu = B.nu[inst];
    B.pobj[inst] = pobj;
    B.dobj[inst] = dobj;
    B.gap[inst] = a.sz;
    B.mu[inst] = nu > 0 ? a.sz / nu : 0.0;
    B.res[3 * inst] = a.rx;
    B.res[3 * inst + 1] = a.ry;
    B.res[3 * inst + 2] = a.rz;
    const double vals[] = {pobj, dobj, a.sz, a.rx, a.ry, a.rz, a.Px, a.Aty, a.Gtz, a.Ax, a.Gx, a.s};
    bool finite = true;
    for (double v : vals) finite = finite && isfinite(v);
    auto conv = [&](double ea, double er) {
        const bool oy = a.ry <= ea + er * fmax(a.Ax, B.b_inf[inst]);
        const bool oz = a.rz <= ea + er * fmax(a.Gx, fmax(a.s, B.h_inf[inst]));
        const bool ox = a.rx <= ea + er * fmax(fmax(a.Px, a.Aty), fmax(a.Gtz, B.c_inf[inst]));
        const bool og = fabs(a.sz) <= ea + er * fmax(1.0, fmax(fabs(pobj), fabs(dobj)));
        return ox && oy && oz && og;
    };
    const int was = B.conv[inst];
    int now = was;
    if (!was && finite && conv(abstol, reltol)) {
        now = 1;
        B.iters[inst] = iter;
    }
    B.conv[inst] = now;
    B.conv_inacc[inst] = (finite && conv(abstol_inacc, reltol_inacc)) ? 1 : 0;
    B.nonfinite[inst] = finite ? 0 : 1;
}

// all-instance flags for the host's loop test: S.converged = every instance converged,
// S.converged_inacc = every unconverged instance meets the inaccurate tolerances,
// S.nonfinite = some unconverged instance is non-finite; S.gap = largest gap
__global__ void k_batch_flags(BatchView B, IPMScalars* S) {
    __shared__ int sc[32], si[32], sn[32];
    __shared__ double sg[32];
    int all = 1, inacc = 1, bad = 0;
    double g = 0.0;
    for (int i = threadIdx.x; i < B.nb; i += blockDim.x) {
        const int cv = B.conv[i];
        all &= cv;
        inacc &= (cv | B.conv_inacc[i]);
        bad |= (!cv && B.nonfinite[i]);
        g = amax(g, B.gap[i]);
    }
    all = __all_sync(0xffffffffu, all);
    inacc = __all_sync(0xffffffffu, inacc);
    bad = __any_sync(0xffffffffu, bad);
    g = warp_max_nonneg(g);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sc[wid] = all; si[wid] = inacc; sn[wid] = bad; sg[wid] = g; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            all &= sc[w]; inacc &= si[w]; bad |= sn[w]; g = fmax(g, sg[w]);
        }
        S->converged = all;
        S->converged_inacc = inacc;
        S->nonfinite = bad;
        S->gap = g;
    }
}

// per-item (orthant entry, then SOC) values of a cone reduction
// mode 0: max step of (u1, du1) and (u2, du2) (min of the two, +inf when unbounded)
// mode 1: shift measure of u1 → out[item], of u2 → out[nitems + item]
__global__ void k_batch_items(ConeView c, ConeGrid g, int mode, const double* __restrict__ u1,
                              const double* __restrict__ du1, const double* __restrict__ u2,
                              const double* __restrict__ du2, double* __restrict__ out) {
    ConeItem it;
    if (!cone_item(c, g, &it)) return;
    const int nitems = c.l + c.nsoc;
    if (it.kind == 0) {
        const int i = it.idx;
        if (mode == 0) {
            double a = INFINITY;
            if (du1[i] < 0.0) a = fmin(a, -u1[i] / du1[i]);
            if (du2[i] < 0.0) a = fmin(a, -u2[i] / du2[i]);
            out[i] = a;
        } else {
            out[i] = -u1[i];
            out[nitems + i] = -u2[i];
        }
        return;
    }
    const int k = it.idx, o = c.off[k], d = c.dim[k];
    const int item = c.l + k;
    if (mode == 0) {
        double a;
        if (it.kind == 1) a = fmin(soc_step<1>(o, d, 0, u1, du1), soc_step<1>(o, d, 0, u2, du2));
        else a = fmin(soc_step<32>(o, d, it.lane, u1, du1), soc_step<32>(o, d, it.lane, u2, du2));
        if (it.lane == 0) out[item] = a;
    } else {
        const int G = it.kind == 1 ? 1 : 32;
        double a1 = 0.0, a2 = 0.0;
        for (int a = 1 + it.lane; a < d; a += G) {
            a1 += u1[o + a] * u1[o + a];
            a2 += u2[o + a] * u2[o + a];
        }
        if (G == 32) { a1 = warp_sum(a1); a2 = warp_sum(a2); }
        if (it.lane == 0) {
            out[item] = sqrt(a1) - u1[o];
            out[nitems + item] = sqrt(a2) - u2[o];
        }
    }
}

// per instance (one warp): min (mode 0) or max (mode 1, two arrays) over its items
__global__ void k_batch_items_reduce(BatchView B, int l, int nsoc, int mode, const double* __restrict__ items,
                                     double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int inst = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (inst >= B.nb) return;
    const int nitems = l + nsoc;
    for (int v = 0; v < (mode == 0 ? 1 : 2); ++v) {
        const double* it = items + (int64_t)v * nitems;
        double a = mode == 0 ? INFINITY : -INFINITY;
        for (int seg = 0; seg < 2; ++seg) {
            const int lo = seg == 0 ? B.lo[inst] : l + B.ko[inst];
            const int hi = seg == 0 ? B.lo[inst + 1] : l + B.ko[inst + 1];
            for (int i = lo + lane; i < hi; i += 32) a = mode == 0 ? fmin(a, it[i]) : fmax(a, it[i]);
        }
        a = mode == 0 ? warp_min(a) : -warp_min(-a);
        if (lane == 0) out[(int64_t)v * B.nb + inst] = a;
    }
}

// u += (1 + α_inst) e where α_inst ≥ 0 (per item of u's instance)
__global__ void k_batch_shift_apply(ConeView c, double* u, const double* __restrict__ alpha) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < c.l) {
        const double a = alpha[c.inst_orth[t]];
        if (a >= 0.0) u[t] += 1.0 + a;
    } else if (t < c.l + c.nsoc) {
        const int k = t - c.l;
        const double a = alpha[c.inst_soc[k]];
        if (a >= 0.0) u[c.off[k]] += 1.0 + a;
    }
}

__global__ void k_batch_sigma(BatchView B, double exponent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.nb) return;
    const double aa = fmin(1.0, B.alpha_max[i]);
    const double sg = pow(1.0 - aa, exponent);
    B.sigma_mu[i] = sg * B.mu[i];
}

__global__ void k_batch_alpha(BatchView B, double step_fraction) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B.nb) return;
    B.alpha[i] = B.conv[i] ? 0.0 : fmin(1.0, step_fraction * B.alpha_max[i]);
}

__global__ void k_batch_update(BatchView B, double* xyz, double* s, const double* __restrict__ d,
                               const double* __restrict__ ds, int N, int nzoff, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) xyz[i] += B.alpha[B.inst_row[i]] * d[i];
    if (i < m) s[i] += B.alpha[B.inst_row[nzoff + i]] * ds[i];
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int launch_batch_residual(const KKTView& K, const BatchView& B, int L, const double* xyz, const double* s,
                          const double* c, const double* b, const double* h, double* r, double* aux, int iter,
                          const IPMScalars& tol, IPMScalars* S, cudaStream_t st) {
    if (K.N) k_batch_residual<<<blocks_for(K.N, 256), 256, 0, st>>>(K, xyz, s, c, b, h, r, aux);
    k_batch_reduce<<<blocks_for((int64_t)B.nb * 32, 256), 256, 0, st>>>(
        B, K.n, K.p, L, xyz, s, c, b, h, r, aux, iter, tol.abstol, tol.reltol, tol.abstol_inacc, tol.reltol_inacc);
    k_batch_flags<<<1, 1024, 0, st>>>(B, S);
    return 3;
}

int launch_batch_max_step(const ConeView& c, const BatchView& B, const double* u1, const double* du1,
                          const double* u2, const double* du2, double* items, cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (!g.blocks()) return 0;
    k_batch_items<<<g.blocks(), kConeThreads, 0, st>>>(c, g, 0, u1, du1, u2, du2, items);
    k_batch_items_reduce<<<blocks_for((int64_t)B.nb * 32, 256), 256, 0, st>>>(B, c.l, c.nsoc, 0, items,
                                                                              B.alpha_max);
    return 2;
}

int launch_batch_shift(const ConeView& c, const BatchView& B, double* s, double* z, double* items,
                       double* shift2, cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (!g.blocks()) return 0;
    k_batch_items<<<g.blocks(), kConeThreads, 0, st>>>(c, g, 1, s, nullptr, z, nullptr, items);
    k_batch_items_reduce<<<blocks_for((int64_t)B.nb * 32, 256), 256, 0, st>>>(B, c.l, c.nsoc, 1, items, shift2);
    const int n = c.l + c.nsoc;
    k_batch_shift_apply<<<blocks_for(n, 256), 256, 0, st>>>(c, s, shift2);
    k_batch_shift_apply<<<blocks_for(n, 256), 256, 0, st>>>(c, z, shift2 + B.nb);
    return 4;
}

int launch_batch_sigma(const BatchView& B, cudaStream_t st) {
    k_batch_sigma<<<blocks_for(B.nb, 256), 256, 0, st>>>(B, 3.0);
    return 1;
}

int launch_batch_step(const BatchView& B, double step_fraction, double* xyz, double* s, const double* d,
                      const double* ds, int N, int nzoff, int m, cudaStream_t st) {
    k_batch_alpha<<<blocks_for(B.nb, 256), 256, 0, st>>>(B, step_fraction);
    k_batch_update<<<blocks_for(N > m ? N : m, 256), 256, 0, st>>>(B, xyz, s, d, ds, N, nzoff, m);
    return 2;
}

}  // namespace qoco
