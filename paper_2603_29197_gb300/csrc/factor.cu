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
#include "fronts.cuh"

#include "qoco_gpu.h"

namespace qoco {

__global__ void __launch_bounds__(128) k_thread_factor(const int* __restrict__ list, int n, FactorView a,
                                                       const double* __restrict__ kval) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && !(a.skip && a.skip[list[t]])) thread_factor_front(list[t], a, kval, NoWait());
}
__global__ void __launch_bounds__(128) k_thread_fwd(const int* __restrict__ list, int n, FactorView a,
                                                    const double* __restrict__ rhs, double* __restrict__ w) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) thread_fwd_front(list[t], a, rhs, w, NoWait());
}
__global__ void __launch_bounds__(128) k_thread_bwd(const int* __restrict__ list, int n, FactorView a,
                                                    const double* __restrict__ w, double* __restrict__ xp,
                                                    double* __restrict__ x, int accumulate) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) thread_bwd_front(list[t], a, w, xp, x, accumulate, NoWait());
}


// One front factored by a whole CTA.  F is the front (shared memory, or the front's
// global slot G itself), lk the W panel (kPanel·f) followed by the broadcast slot and
// the pivot signs.  wait() must be called by every thread.
template <class Wait>
__device__ __forceinline__ bool cta_factor_front(int s, const FactorView& a, const double* __restrict__ kval,
                                                 double* F, double* lk, bool in_smem, const Wait& wait) {
    const int f = a.nrow[s], c = a.ncol[s], first = a.first[s];
    double* G = a.front + a.front_off[s];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t ff = (int64_t)f * f;
    for (int64_t i = tid; i < ff; i += nt) F[i] = 0.0;
    __syncthreads();
    for (int64_t e = a.amap_ptr[s] + tid; e < a.amap_ptr[s + 1]; e += nt) {
        const int off = (int)a.amap_off[e];
        double v = kval[a.amap_slot[e]];
        const int col = off / f, row = off - col * f;
        if (row == col) v += a.dsign[first + col] > 0 ? a.eps : -a.eps;
        F[off] = v;
    }
    __syncthreads();
    const int k0 = a.child_ptr[s], nch = a.child_ptr[s + 1] - k0;
    // the first 32 child records, fetched by warp 0 before the wait and broadcast through
    // a small shared table
    __shared__ ChildInfo s_ci[32];
    if (tid < nch && tid < 32) s_ci[tid] = a.cinfo[k0 + tid];
    stage_pivot_signs(lk + (size_t)kPanel * f, c, first, a, tid, nt);
    __syncthreads();
    if (!wait()) return false;
    extend_add_children<false, 12, double>(F, f, a, nch, [&](int k) { return k < 32 ? s_ci[k] : a.cinfo[k0 + k]; },
                                          tid, nt);
    const int nreg = blocked_ldlt<false>(F, lk, lk + (size_t)kPanel * f, f, c, first, a, tid, nt);
    if (nreg) atomicAdd(a.nreg, nreg);  // the pivot thread's count
    if (in_smem)
        for (int64_t i = tid; i < ff; i += nt) G[i] = F[i];
    __syncthreads();
    return true;
}

// One CTA per front of a level.  Dynamic shared memory: the front (f² doubles, SMEM
// variant), then the W panel, broadcast slot and pivot signs.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_front_factor(const int* __restrict__ list, FactorView a,
                                                      const double* __restrict__ kval) {
    extern __shared__ double smem[];
    const int s = list[blockIdx.x];
    if (a.skip && a.skip[s]) return;  // a leaf-group member (whole CTA)
    const int f = a.nrow[s];
    double* F = SMEM ? smem : a.front + a.front_off[s];
    double* lk = SMEM ? smem + (size_t)f * f : smem;
    cta_factor_front(s, a, kval, F, lk, SMEM, NoWait());
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

// one warp per listed supernode of a level
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_warp_factor(const int* __restrict__ list, int n,
                                                                    FactorView a, const double* __restrict__ kval,
                                                                    int fmax) {
    extern __shared__ double smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kWarpsPerBlock + wid;
    if (t >= n || (a.skip && a.skip[list[t]])) return;
    double* F = smem + (size_t)wid * wfactor_stride(fmax);
    warp_factor_front(list[t], a, kval, F, F + fmax * fmax, lane, NoWait());
}
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_warp_fwd(const int* __restrict__ list, int n,
                                                                 FactorView a, const double* __restrict__ rhs,
                                                                 double* __restrict__ w, int fmax) {
    extern __shared__ double smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * kWarpsPerBlock + wid;
    if (t >= n) return;
    double* v = smem + (size_t)wid * fmax * (fmax + 1);
    warp_fwd_front(list[t], a, rhs, w, v, v + fmax, lane, NoWait());
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
    warp_bwd_front(list[t], a, w, xp, x, accumulate, v, v + fmax, lane, NoWait());
}

// ---------------------------------------------------------------------------
// Dataflow solve: one launch, no barriers.  Work items (warp fronts and batches of 32
// one-thread fronts) are handed out by an atomic counter: first the forward items in
// level order, then the backward items in reverse order.  A forward item waits until
// its fronts' children have finished their forward step; a backward item waits for
// its parent's backward step (a root for its own forward step).  Since every item
// only waits on items handed out before it, which are owned by running warps, the
// scheme cannot deadlock and needs no co-residency.  Flags hold the launch's epoch
// (no reset between launches); producers fence before raising a flag, consumers fence
// after seeing it and read the produced data through L2 (__ldcg).  Every wait polls a
// bounded number of times, then raises the error flag; all warps then leave.
// ---------------------------------------------------------------------------
constexpr int kDataflowThreads = 128;

__device__ __forceinline__ bool wait_epoch(const int* flag, int epoch, int* err, long long max_spins) {
    const volatile int* vf = flag;
    const volatile int* ve = err;
    long long spins = 0;
    while (*vf != epoch) {
        if (*ve) return false;
        if (++spins > max_spins) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// Self-test of the dataflow wait's timeout path: warp 0 of the probe waits on a flag that
// no item ever publishes, so its wait gives up after max_spins polls and raises the error
// flag; warp 1 waits on the same flag and leaves as soon as it sees that error, as every
// dataflow warp does.
__global__ void k_wait_timeout_probe(const int* flag, int* err, long long max_spins) {
    if ((threadIdx.x & 31) == 0) wait_epoch(flag, 1, err, max_spins);
}

int selftest_wait_timeout(long long max_spins, cudaStream_t st) {
    int* buf = nullptr;
    QOCO_CUDA_TRY(cudaMalloc((void**)&buf, 2 * sizeof(int)));
    int rc = 0, err = 0;
    cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) {
        k_wait_timeout_probe<<<1, 64, 0, st>>>(buf, buf + 1, max_spins);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "wait self-test", __FILE__, __LINE__);
    else rc = err ? QOCO_GPU_ERR_DEVICE_TIMEOUT : 0;
    cudaFree(buf);
    return rc;
}

__global__ void __launch_bounds__(kDataflowThreads) k_solve_dataflow(
    const int* __restrict__ items, int nitems, const int* __restrict__ tb_ptr, const int* __restrict__ sthread,
    FactorView a, const double* __restrict__ rhs, double* w, double* xp, double* x, int accumulate, int fmax,
    int* fdone, int* bdone, DataflowState ds, int it0) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* v = smem + (size_t)wid * fmax * (fmax + 1);
    double* P = v + fmax;
    for (;;) {
        int it = 0, stop = 0;
        if (lane == 0) {
            it = (int)atomicAdd(ds.next, 1u) + it0;
            stop = *(volatile int*)ds.err;
        }
        it = __shfl_sync(0xffffffffu, it, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (stop || it >= 2 * nitems) return;
        const bool fwd = it < nitems;
        const int item = fwd ? items[it] : items[2 * nitems - 1 - it];
        int* done = fwd ? fdone : bdone;
        if (item >= 0) {
            const int s = item;
            // warp-wide wait: lanes share the children (forward) or lane 0 waits for the
            // parent (backward); every lane then fences before the dependent loads
            auto wait = [&]() {
                bool ok = true;
                if (fwd) {
                    for (int k = a.child_ptr[s] + lane; k < a.child_ptr[s + 1]; k += 32)
                        ok = ok && wait_epoch(fdone + a.child[k], ds.epoch, ds.err, ds.max_spins);
                } else if (lane == 0) {
                    const int p = a.parent[s];
                    ok = wait_epoch(p >= 0 ? bdone + p : fdone + s, ds.epoch, ds.err, ds.max_spins);
                }
                ok = __all_sync(0xffffffffu, ok);
                __threadfence();
                return ok;
            };
            const bool ok = fwd ? warp_fwd_front(s, a, rhs, w, v, P, lane, wait)
                                : warp_bwd_front(s, a, w, xp, x, accumulate, v, P, lane, wait);
            if (!ok) return;
            __threadfence();
            __syncwarp();
            if (lane == 0) atomicExch(done + s, ds.epoch);
        } else {
            const int b = -item - 1;
            const int t = tb_ptr[b] + lane;
            bool ok = true;
            if (t < tb_ptr[b + 1]) {
                const int s = sthread[t];
                auto wait = [&]() {
                    bool good = true;
                    if (fwd) {
                        for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1] && good; ++k)
                            good = wait_epoch(fdone + a.child[k], ds.epoch, ds.err, ds.max_spins);
                    } else {
                        const int p = a.parent[s];
                        good = wait_epoch(p >= 0 ? bdone + p : fdone + s, ds.epoch, ds.err, ds.max_spins);
                    }
                    __threadfence();
                    return good;
                };
                ok = fwd ? thread_fwd_front(s, a, rhs, w, wait) : thread_bwd_front(s, a, w, xp, x, accumulate, wait);
                if (ok) {
                    __threadfence();
                    atomicExch(done + s, ds.epoch);
                }
            }
            if (!__all_sync(0xffffffffu, ok)) return;
        }
    }
}

static size_t dataflow_smem(int fmax) {
    return (size_t)(kDataflowThreads / 32) * fmax * (fmax + 1) * sizeof(double);
}

int plan_dataflow_solve(FactorPlan& P, int max_warp_f, bool any_cta_front) {
    P.dataflow = false;
    if (any_cta_front || P.nitems == 0) return 0;
    const int fmax = max(1, max_warp_f);
    const size_t sm = dataflow_smem(fmax);
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_solve_dataflow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int dev = 0, nsm = 0, occ = 0;
    QOCO_CUDA_TRY(cudaGetDevice(&dev));
    QOCO_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    QOCO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve_dataflow, kDataflowThreads, sm));
    if (occ < 1) return 0;
    P.dataflow = true;
    P.dataflow_grid = nsm * occ;
    P.dataflow_fmax = fmax;
    return 0;
}

int launch_solve_dataflow(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                          double* x, bool accumulate, const DataflowState& ds, cudaStream_t st, bool bwd_only) {
    QOCO_CUDA_TRY(cudaMemsetAsync(ds.next, 0, sizeof(unsigned int), st));
    k_solve_dataflow<<<P.dataflow_grid, kDataflowThreads, dataflow_smem(P.dataflow_fmax), st>>>(
        P.d_items, P.nitems, P.d_tb_ptr, P.d_sthread, a, rhs, w, xp, x, accumulate ? 1 : 0, P.dataflow_fmax,
        P.d_fdone, P.d_bdone, ds, bwd_only ? P.nitems : 0);
    return 1;
}

// The fused forward step of front s (order ≤ kWarpFront) by one warp, after its
// factorisation has been published: it waits (bounded) for its children's forward steps,
// then runs with F holding the factored front (leading dimension f) and v free shared
// memory of at least f doubles.  The same arithmetic as the dataflow solve's step for a
// front of this order (one thread up to kThreadFront, else one warp), so a fused forward
// sweep gives the same bits as a separate one.
__device__ __forceinline__ bool fused_fwd_warp(int s, const FactorView& a, const FwdFuse& fz, const DataflowState& ds,
                                               const double* F, double* v, int lane) {
    if (a.nrow[s] <= kThreadFront) {
        bool ok = true;
        if (lane == 0) {
            auto wait = [&]() {
                bool good = true;
                for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1] && good; ++k)
                    good = wait_epoch(fz.fdone + a.child[k], fz.epoch, ds.err, ds.max_spins);
                __threadfence();
                return good;
            };
            ok = thread_fwd_front(s, a, fz.rhs, fz.w, wait);
        }
        return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    }
    auto wait = [&]() {
        bool good = true;
        for (int k = a.child_ptr[s] + lane; k < a.child_ptr[s + 1]; k += 32)
            good = good && wait_epoch(fz.fdone + a.child[k], fz.epoch, ds.err, ds.max_spins);
        good = __all_sync(0xffffffffu, good);
        __threadfence();
        return good;
    };
    return warp_fwd_front<decltype(wait), 8, false>(s, a, fz.rhs, fz.w, v, F, lane, wait);
}

// Shared memory per warp of the dataflow factorisation: one front of order ≤ fmax, or two
// of order ≤ kPairFront (one per half-warp).
__host__ __device__ __forceinline__ int fdataflow_warp_stride(int fmax) {
    const int pf = fmax < kPairFront ? fmax : kPairFront;
    const int one = wfactor_stride(fmax), two = 2 * wfactor_stride(pf);
    return one > two ? one : two;
}

// ---------------------------------------------------------------------------
// Dataflow factorisation: one launch, blocks of kDataflowThreads take items in level
// order from an atomic counter.  Item kinds (low two bits): 0 = batch of up to 128
// one-thread fronts, 1 = group of up to 4 warp fronts, 2 = one front for the whole
// CTA, 3 = group of up to 8 fronts of order ≤ kPairFront, two per warp (one per
// half-warp).  A front waits (bounded polls) for its children's completion flags after its
// independent assembly; the deadlock argument is the one of the dataflow solve.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kDataflowThreads) k_factor_dataflow(
    const int* __restrict__ items, int nitems, const int* __restrict__ tb_ptr, const int* __restrict__ tlist,
    const int* __restrict__ wg_ptr, const int* __restrict__ wlist, FactorView a, const double* __restrict__ kval,
    int fmax, int* cdone, DataflowState ds, FwdFuse fz) {
    extern __shared__ double smem[];
    __shared__ int s_it, s_stop;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            s_it = (int)atomicAdd(ds.next, 1u);
            s_stop = *(volatile int*)ds.err;
        }
        __syncthreads();
        const int it = s_it, stop = s_stop;
        __syncthreads();
        if (stop || it >= nitems) return;
        const int item = items[it];
        const int kind = item & 3, idx = item >> 2;
        bool ok = true;
        if (kind == 0) {
            const int t = tb_ptr[idx] + threadIdx.x;
            if (t < tb_ptr[idx + 1]) {
                const int s = tlist[t];
                auto wait = [&]() {
                    bool good = true;
                    for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1] && good; ++k)
                        good = wait_epoch(cdone + a.child[k], ds.epoch, ds.err, ds.max_spins);
                    __threadfence();
                    return good;
                };
                ok = thread_factor_front(s, a, kval, wait);
                if (ok) {
                    __threadfence();
                    atomicExch(cdone + s, ds.epoch);
                }
                // the fused forward step, after the factor is published: the parent's
                // factorisation does not wait for it
                if (ok && fz.rhs) {
                    auto fwait = [&]() {
                        bool good = true;
                        for (int k = a.child_ptr[s]; k < a.child_ptr[s + 1] && good; ++k)
                            good = wait_epoch(fz.fdone + a.child[k], fz.epoch, ds.err, ds.max_spins);
                        __threadfence();
                        return good;
                    };
                    ok = thread_fwd_front(s, a, fz.rhs, fz.w, fwait);
                    if (ok) {
                        __threadfence();
                        atomicExch(fz.fdone + s, fz.epoch);
                    }
                }
            }
        } else if (kind == 1) {
            const int t = wg_ptr[idx] + wid;
            if (t < wg_ptr[idx + 1]) {
                const int s = wlist[t];
                double* F = smem + (size_t)wid * fdataflow_warp_stride(fmax);
                auto wait = [&]() {
                    bool good = true;
                    for (int k = a.child_ptr[s] + lane; k < a.child_ptr[s + 1]; k += 32)
                        good = good && wait_epoch(cdone + a.child[k], ds.epoch, ds.err, ds.max_spins);
                    good = __all_sync(0xffffffffu, good);
                    __threadfence();
                    return good;
                };
                ok = warp_factor_front(s, a, kval, F, F + fmax * fmax, lane, wait);
                if (ok) {
                    __threadfence();
                    __syncwarp();
                    if (lane == 0) atomicExch(cdone + s, ds.epoch);
                }
                if (ok && fz.rhs) {
                    ok = fused_fwd_warp(s, a, fz, ds, F, F + fmax * fmax, lane);
                    if (ok) {
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) atomicExch(fz.fdone + s, fz.epoch);
                    }
                }
            }
        } else if (kind == 3) {
            // two fronts of order ≤ kPairFront per warp, one per half (lanes 0–15, 16–31)
            const int h = lane >> 4, hl = lane & 15;
            const int pf = min(fmax, kPairFront);
            const unsigned hmask = 0xffffu << (16 * h);
            double* Fw = smem + (size_t)wid * fdataflow_warp_stride(fmax);
            const int t = wg_ptr[idx] + 2 * wid + h;
            bool good = true;
            if (t < wg_ptr[idx + 1]) {
                const int s = wlist[t];
                double* F = Fw + (size_t)h * wfactor_stride(pf);
                auto wait = [&]() {
                    bool g2 = true;
                    for (int k = a.child_ptr[s] + hl; k < a.child_ptr[s + 1]; k += 16)
                        g2 = g2 && wait_epoch(cdone + a.child[k], ds.epoch, ds.err, ds.max_spins);
                    g2 = __all_sync(hmask, g2);
                    __threadfence();
                    return g2;
                };
                good = warp_factor_front<decltype(wait), double, 8, 16>(s, a, kval, F, F + pf * pf, lane, wait);
                if (good) {
                    __threadfence();
                    __syncwarp(hmask);
                    if (hl == 0) atomicExch(cdone + s, ds.epoch);
                }
            }
            __syncwarp();
            // the fused forward steps of the two fronts, one after the other by the whole warp
            if (fz.rhs) {
                for (int hh = 0; hh < 2; ++hh) {
                    const int th = wg_ptr[idx] + 2 * wid + hh;
                    if (th >= wg_ptr[idx + 1]) break;
                    if (__shfl_sync(0xffffffffu, good ? 1 : 0, 16 * hh) == 0) continue;
                    const int sh = wlist[th];
                    double* Fh = Fw + (size_t)hh * wfactor_stride(pf);
                    const bool g3 = fused_fwd_warp(sh, a, fz, ds, Fh, Fh + pf * pf, lane);
                    if (g3) {
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) atomicExch(fz.fdone + sh, fz.epoch);
                    } else {
                        good = false;
                    }
                }
            }
            ok = good;
        } else {
            const int s = idx;
            const int f = a.nrow[s];
            auto wait = [&]() {
                bool good = true;
                for (int k = a.child_ptr[s] + (int)threadIdx.x; k < a.child_ptr[s + 1]; k += blockDim.x)
                    good = good && wait_epoch(cdone + a.child[k], ds.epoch, ds.err, ds.max_spins);
                good = __syncthreads_and(good) != 0;
                __threadfence();
                return good;
            };
            ok = cta_factor_front(s, a, kval, smem, smem + (size_t)f * f, true, wait);
            if (ok) {
                __threadfence();
                if (threadIdx.x == 0) atomicExch(cdone + s, ds.epoch);
            }
            if (ok && fz.rhs) {
                bool good = true;
                if (wid == 0) good = fused_fwd_warp(s, a, fz, ds, smem, smem + (size_t)f * f, lane);
                ok = __syncthreads_and(good) != 0;
                if (ok) {
                    __threadfence();
                    if (threadIdx.x == 0) atomicExch(fz.fdone + s, fz.epoch);
                }
            }
        }
        if (!__syncthreads_and(ok)) return;
    }
}

static size_t fdataflow_smem(int fmax) {
    return (size_t)(kDataflowThreads / 32) * fdataflow_warp_stride(fmax) * sizeof(double);
}

int plan_dataflow_factor(FactorPlan& P, int fmax, bool any_large) {
    P.fdataflow = false;
    if (any_large || P.nfitems == 0 || fmax > kWarpFront) return 0;
    fmax = max(fmax, 1);
    const size_t sm = fdataflow_smem(fmax);
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_factor_dataflow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int dev = 0, nsm = 0, occ = 0;
    QOCO_CUDA_TRY(cudaGetDevice(&dev));
    QOCO_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    QOCO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_factor_dataflow, kDataflowThreads, sm));
    if (occ < 1) return 0;
    P.fdataflow = true;
    P.fdataflow_grid = nsm * occ;
    P.fdataflow_fmax = fmax;
    return 0;
}

int launch_factor_dataflow(const FactorPlan& P, const FactorView& a, const double* kval, const DataflowState& ds,
                           cudaStream_t st, const FwdFuse& fz) {
    QOCO_CUDA_TRY(cudaMemsetAsync(ds.next, 0, sizeof(unsigned int), st));
    k_factor_dataflow<<<P.fdataflow_grid, kDataflowThreads, fdataflow_smem(P.fdataflow_fmax), st>>>(
        P.d_fitems, P.nfitems, P.d_ftb_ptr, P.d_thread, P.d_fwg_ptr, P.d_warp, a, kval, P.fdataflow_fmax,
        P.d_cdone, ds, fz);
    return 1;
}

// ---------------------------------------------------------------------------
// Batches: one CTA per instance.  A persistent grid takes instances from a queue that
// holds the largest first; the CTA walks the instance's tree level by level (thread
// fronts and warp fronts of a level side by side, a block barrier between levels), so
// no flag or cross-CTA wait is involved and a front's children are complete, and
// visible to the whole CTA, when it starts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int inst_take(unsigned int* next) {
    __shared__ int s_i;
    if (threadIdx.x == 0) s_i = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int i = s_i;
    __syncthreads();
    return i;
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) k_inst_factor(const int* __restrict__ order, int ninst,
                                                         const int* __restrict__ lv_ptr, const int* __restrict__ ent,
                                                         const int* __restrict__ sched, FactorView a,
                                                         const double* __restrict__ kval, int fmax,
                                                         unsigned int* next) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* F = smem + (size_t)wid * wfactor_stride(fmax);
    for (;;) {
        const int i = inst_take(next);
        if (i >= ninst) return;
        const int inst = order[i];
        for (int k = lv_ptr[inst]; k < lv_ptr[inst + 1]; ++k) {
            const int t0 = ent[3 * k], w0 = ent[3 * k + 1], e1 = ent[3 * k + 2];
            for (int t = t0 + (int)threadIdx.x; t < w0; t += NW * 32) thread_factor_front(sched[t], a, kval, NoWait());
            for (int t = w0 + wid; t < e1; t += NW) warp_factor_front(sched[t], a, kval, F, F + fmax * fmax, lane, NoWait());
            __syncthreads();
        }
    }
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) k_inst_solve(const int* __restrict__ order, int ninst,
                                                        const int* __restrict__ lv_ptr, const int* __restrict__ ent,
                                                        const int* __restrict__ sched, FactorView a,
                                                        const double* __restrict__ rhs, double* w, double* xp,
                                                        double* x, int accumulate, int fmax, unsigned int* next) {
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double* v = smem + (size_t)wid * fmax * (fmax + 1);
    double* P = v + fmax;
    for (;;) {
        const int i = inst_take(next);
        if (i >= ninst) return;
        const int inst = order[i], k0 = lv_ptr[inst], k1 = lv_ptr[inst + 1];
        for (int k = k0; k < k1; ++k) {
            const int t0 = ent[3 * k], w0 = ent[3 * k + 1], e1 = ent[3 * k + 2];
            for (int t = t0 + (int)threadIdx.x; t < w0; t += NW * 32) thread_fwd_front(sched[t], a, rhs, w, NoWait());
            for (int t = w0 + wid; t < e1; t += NW) warp_fwd_front(sched[t], a, rhs, w, v, P, lane, NoWait());
            __syncthreads();
        }
        for (int k = k1 - 1; k >= k0; --k) {
            const int t0 = ent[3 * k], w0 = ent[3 * k + 1], e1 = ent[3 * k + 2];
            for (int t = t0 + (int)threadIdx.x; t < w0; t += NW * 32)
                thread_bwd_front(sched[t], a, w, xp, x, accumulate, NoWait());
            for (int t = w0 + wid; t < e1; t += NW) warp_bwd_front(sched[t], a, w, xp, x, accumulate, v, P, lane, NoWait());
            __syncthreads();
        }
    }
}

static size_t inst_factor_smem(int nw, int fmax) { return (size_t)nw * wfactor_stride(fmax) * sizeof(double); }
static size_t inst_solve_smem(int nw, int fmax) { return (size_t)nw * fmax * (fmax + 1) * sizeof(double); }

int plan_instances(FactorPlan& P, int fmax) {
    fmax = max(fmax, 1);
    int dev = 0, nsm = 0;
    QOCO_CUDA_TRY(cudaGetDevice(&dev));
    QOCO_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const void* fk[2] = {(const void*)k_inst_factor<4>, (const void*)k_inst_factor<8>};
    const void* sk[2] = {(const void*)k_inst_solve<4>, (const void*)k_inst_solve<8>};
    for (int v = 0; v < 2; ++v) {
        const int nw = v ? 8 : 4;
        const size_t fs = inst_factor_smem(nw, fmax), ss = inst_solve_smem(nw, fmax);
        QOCO_CUDA_TRY(cudaFuncSetAttribute(fk[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs));
        QOCO_CUDA_TRY(cudaFuncSetAttribute(sk[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss));
        int of = 0, os = 0;
        QOCO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, fk[v], nw * 32, fs));
        QOCO_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&os, sk[v], nw * 32, ss));
        if (of < 1 || os < 1) return 0;
        P.inst_fgrid[v] = min(nsm * of, P.ninst);
        P.inst_sgrid[v] = min(nsm * os, P.ninst);
    }
    P.inst_fmax = fmax;
    P.inst = true;
    return 0;
}

// variant 1–4: bit 0 of (variant − 1) = 8 warps, bit 1 = every front one warp
int launch_inst_factor(const FactorPlan& P, const FactorView& a, const double* kval, int variant,
                       cudaStream_t st) {
    const int v8 = (variant - 1) & 1;
    const FactorPlan::InstSched& I = P.isched[((variant - 1) >> 1) & 1];
    QOCO_CUDA_TRY(cudaMemsetAsync(P.d_inst_next, 0, sizeof(unsigned int), st));
    if (v8)
        k_inst_factor<8><<<P.inst_fgrid[1], 256, inst_factor_smem(8, P.inst_fmax), st>>>(
            P.d_inst_order, P.ninst, I.d_lv_ptr, I.d_ent, I.d_sched, a, kval, P.inst_fmax, P.d_inst_next);
    else
        k_inst_factor<4><<<P.inst_fgrid[0], 128, inst_factor_smem(4, P.inst_fmax), st>>>(
            P.d_inst_order, P.ninst, I.d_lv_ptr, I.d_ent, I.d_sched, a, kval, P.inst_fmax, P.d_inst_next);
    return 1;
}

int launch_inst_solve(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                      double* x, bool accumulate, int variant, cudaStream_t st) {
    const int v8 = (variant - 1) & 1;
    const FactorPlan::InstSched& I = P.isched[((variant - 1) >> 1) & 1];
    unsigned int* next = P.d_inst_next + 1;
    QOCO_CUDA_TRY(cudaMemsetAsync(next, 0, sizeof(unsigned int), st));
    const int acc = accumulate ? 1 : 0;
    if (v8)
        k_inst_solve<8><<<P.inst_sgrid[1], 256, inst_solve_smem(8, P.inst_fmax), st>>>(
            P.d_inst_order, P.ninst, I.d_lv_ptr, I.d_ent, I.d_sched, a, rhs, w, xp, x, acc, P.inst_fmax, next);
    else
        k_inst_solve<4><<<P.inst_sgrid[0], 128, inst_solve_smem(4, P.inst_fmax), st>>>(
            P.d_inst_order, P.ninst, I.d_lv_ptr, I.d_ent, I.d_sched, a, rhs, w, xp, x, acc, P.inst_fmax, next);
    return 1;
}

// ---- launchers ----------------------------------------------------------------
static int wblocks(int n) { return (n + kWarpsPerBlock - 1) / kWarpsPerBlock; }
// per warp: the front vector (fmax) and the panel (≤ fmax·fmax)
static size_t wsolve_smem(int fmax) { return (size_t)kWarpsPerBlock * fmax * (fmax + 1) * sizeof(double); }
static size_t wfactor_smem(int fmax) { return (size_t)kWarpsPerBlock * wfactor_stride(fmax) * sizeof(double); }

int launch_factor(const FactorPlan& P, const FactorView& a, const double* kval, cudaStream_t st) {
    int launches = 0;
    if (!P.groups.empty()) launches += launch_leaf_groups(P, a, kval, st);
    for (int lv = 0; lv < (int)P.levels.size(); ++lv) {
        const LevelPlan& L = P.levels[lv];
        if (L.n_thread) {
            k_thread_factor<<<(L.n_thread + 127) / 128, 128, 0, st>>>(P.d_thread + L.off_thread, L.n_thread, a, kval);
            ++launches;
        }
        if (L.n_warp) {
            const int fm = L.max_warp_f;
            k_warp_factor<<<wblocks(L.n_warp), kWarpsPerBlock * 32, wfactor_smem(fm), st>>>(
                P.d_warp + L.off_warp, L.n_warp, a, kval, fm);
            ++launches;
        }
        if (L.n_small) {
            const size_t sm = ((size_t)L.max_small * (L.max_small + kPanel + 1) + kPanel + 1) * sizeof(double);
            const int threads = L.max_small <= 64 ? 128 : 256;
            k_front_factor<true><<<L.n_small, threads, sm, st>>>(P.d_small + L.off_small, a, kval);
            ++launches;
        }
        if (L.n_large) {
            const size_t sm = ((size_t)(kPanel + 1) * L.max_large_f + kPanel + 1) * sizeof(double);
            k_front_factor<false><<<L.n_large, 256, sm, st>>>(P.d_large + L.off_large, a, kval);
            ++launches;
        }
        for (int t = 0; t < L.n_big; ++t) launches += launch_big_factor(P, a, kval, L.off_big + t, st);
    }
    return launches;
}

int launch_solve(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                 double* x, bool accumulate, cudaStream_t st) {
    int launches = 0;
    const int nl = (int)P.levels.size();
    const int acc = accumulate ? 1 : 0;
    for (int lv = 0; lv < nl; ++lv) {
        const LevelPlan& L = P.levels[lv];
        if (L.n_sthread) {
            k_thread_fwd<<<(L.n_sthread + 127) / 128, 128, 0, st>>>(P.d_sthread + L.off_sthread, L.n_sthread, a,
                                                                   rhs, w);
            ++launches;
        }
        if (L.n_swarp) {
            k_warp_fwd<<<wblocks(L.n_swarp), kWarpsPerBlock * 32, wsolve_smem(L.max_swarp_f), st>>>(
                P.d_swarp + L.off_swarp, L.n_swarp, a, rhs, w, L.max_swarp_f);
            ++launches;
        }
        if (L.n_cta) {
            k_fwd<<<L.n_cta, 128, (size_t)L.max_cta_f * sizeof(double), st>>>(P.d_cta + L.off_cta, a, rhs, w);
            ++launches;
        }
        for (int t = 0; t < L.n_big; ++t) launches += launch_big_fwd(P, a, rhs, w, L.off_big + t, st);
    }
    for (int lv = nl - 1; lv >= 0; --lv) {
        const LevelPlan& L = P.levels[lv];
        if (L.n_sthread) {
            k_thread_bwd<<<(L.n_sthread + 127) / 128, 128, 0, st>>>(P.d_sthread + L.off_sthread, L.n_sthread, a, w,
                                                                   xp, x, acc);
            ++launches;
        }
        if (L.n_swarp) {
            k_warp_bwd<<<wblocks(L.n_swarp), kWarpsPerBlock * 32, wsolve_smem(L.max_swarp_f), st>>>(
                P.d_swarp + L.off_swarp, L.n_swarp, a, w, xp, x, acc, L.max_swarp_f);
            ++launches;
        }
        if (L.n_cta) {
            k_bwd<<<L.n_cta, 128, (size_t)L.max_cta_f * sizeof(double), st>>>(P.d_cta + L.off_cta, a, w, xp, x, acc);
            ++launches;
        }
        for (int t = 0; t < L.n_big; ++t) launches += launch_big_bwd(P, a, w, xp, x, accumulate, L.off_big + t, st);
    }
    return launches;
}

int factor_set_attributes() {
    const int warp_smem = (int)wfactor_smem(kWarpFront);
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_front_factor<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (kSmemFront * (kSmemFront + kPanel + 1) + kPanel + 1) * (int)sizeof(double)));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_front_factor<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ((kPanel + 1) * kMaxFactorFront + kPanel + 1) * (int)sizeof(double)));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_warp_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, warp_smem));
    const int wsolve = kWarpsPerBlock * kWarpFront * (kWarpFront + 1) * (int)sizeof(double);
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_warp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, wsolve));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_warp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, wsolve));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSolveFront * 8));
    QOCO_CUDA_TRY(cudaFuncSetAttribute(k_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSolveFront * 8));
    return 0;
}

}  // namespace qoco
