// Device interior-point driver and the C ABI (include/qoco_gpu.h).
//
// One iteration (paper §2: one factorisation, two solves, cone operations):
//   residuals + stopping test (K6/K8) → NT scaling and −W² into the KKT values
//   (K1/K2) → numeric LDLᵀ (K5) → predictor rhs (K3), solve + refinement (K7/K6),
//   Δs, affine step and σ (K4) → corrector rhs, solve + refinement, Δs, step (K4)
//   → update.  All of it runs on the device; the host reads one small struct of
//   scalars per iteration (the stopping test) and one flag per refinement check.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "batch.h"
#include "batch_ipm.h"
#include "cone_kernels.h"
#include "factor.h"
#include "krylov.h"
#include "plan.h"
#include "qoco_gpu.h"
#include "row_kernels.h"
#include "symbolic.h"

namespace qoco {

static thread_local char g_cuda_msg[160];

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_cuda_msg, sizeof g_cuda_msg, "CUDA error %s at %s:%d (%s)", cudaGetErrorString(e), file,
             line, what);
    if (e == cudaErrorMemoryAllocation) return QOCO_GPU_ERR_OOM;
    return QOCO_GPU_ERR_CUDA;
}

// ---- small vector kernels ---------------------------------------------------------
__global__ void k_init_rhs(double* rhs, const double* c, const double* b, const double* h, int n, int p,
                           int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rhs[i] = -c[i];
    else if (i < n + p) rhs[i] = b[i - n];
    else if (i < n + p + m) rhs[i] = h[i - n - p];
}
// xyz ← sol, s ← −z
__global__ void k_init_iterate(const double* sol, double* xyz, double* s, int n, int p, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n + p + m) xyz[i] = sol[i];
    if (i >= n + p && i < n + p + m) s[i - n - p] = -sol[i];
}
__global__ void k_shift_finalize(const double* partial, int nb, IPMScalars* S) {
    __shared__ double sm[64];
    double a = -INFINITY, b = -INFINITY;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a = fmax(a, partial[2 * i]);
        b = fmax(b, partial[2 * i + 1]);
    }
    a = -warp_min(-a);
    b = -warp_min(-b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sm[wid] = a; sm[32 + wid] = b; }
    __syncthreads();
    if (wid == 0) {
        const bool ok = lane < (int)(blockDim.x >> 5);
        double t1 = ok ? sm[lane] : -INFINITY, t2 = ok ? sm[32 + lane] : -INFINITY;
        t1 = -warp_min(-t1);
        t2 = -warp_min(-t2);
        if (lane == 0) { S->shift[0] = t1; S->shift[1] = t2; }
    }
}
__global__ void k_neg_copy(double* dst, const double* src, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = -src[i];
}
__global__ void k_sigma(IPMScalars* S, double exponent) {
    const double aa = fmin(1.0, S->alpha_max);
    S->alpha_a = aa;
    const double sg = pow(1.0 - aa, exponent);
    S->sigma = sg;
    S->sigma_mu = sg * S->mu;
}
__global__ void k_set(double* p, double v) { *p = v; }
__global__ void k_alpha(IPMScalars* S) { S->alpha = fmin(1.0, S->step_fraction * S->alpha_max); }
__global__ void k_update(double* xyz, double* s, const double* d, const double* ds, const IPMScalars* S,
                         int N, int m) {
    const double a = S->alpha;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) xyz[i] += a * d[i];
    if (i < m) s[i] += a * ds[i];
}


// ---- adjoint and parametric-update kernels ----------------------------------------
// rp = g, plus t2 on the z rows: the exact complementarity block's term s∘(z\v_z),
// moved to the right-hand side so that the plain KKT SpMV gives K̂ᵀ's residual
__global__ void k_adj_rhs(double* rp, const double* g, const double* t2, int np, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) rp[i] = g[i] + (i >= np && t2 ? t2[i - np] : 0.0);
}
__global__ void k_w2_zero(double* kval, const int64_t* slot, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) kval[slot[i]] = 0.0;
}
// ∂L/∂(data entry) for the entry at KKT position (a, b): −(u_a v_b + v_a u_b), halved
// on the diagonal (P_ii); entries [0, nP) are P's, then A's, then G's
__global__ void k_adj_data_grad(const int* __restrict__ ca, const int* __restrict__ cb, int64_t nnz,
                                int64_t nP, int64_t nA, const double* __restrict__ u,
                                const double* __restrict__ v, double* dP, double* dA, double* dG) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    double* out;
    int64_t j;
    if (k < nP) { out = dP; j = k; }
    else if (k < nP + nA) { out = dA; j = k - nP; }
    else { out = dG; j = k - nP - nA; }
    if (!out) return;
    const int a = ca[k], b = cb[k];
    const double gk = -(u[a] * v[b] + v[a] * u[b]);
    out[j] = a == b ? 0.5 * gk : gk;
}
__global__ void k_adj_vec_grad(const double* v, double* dc, double* db, double* dh, int n, int p, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) { if (dc) dc[i] = -v[i]; }
    else if (i < n + p) { if (db) db[i - n] = v[i]; }
    else if (i < n + p + m) { if (dh) dh[i - n - p] = v[i]; }
}
// KKT value slots fed by problem data ← the new values (src indexes [P | A | G])
__global__ void k_scatter_data(double* kval, const int64_t* __restrict__ slot, const int64_t* __restrict__ src,
                               int64_t n, const double* Pv, const double* Av, const double* Gv, int64_t nP,
                               int64_t nA) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t k = src[i];
    const double* p = k < nP ? Pv : k < nP + nA ? Av : Gv;
    const int64_t j = k < nP ? k : k < nP + nA ? k - nP : k - nP - nA;
    if (p) kval[slot[i]] = p[j];
}
// ‖c‖∞, ‖b‖∞, ‖h‖∞ (stopping-test scales) of the current data; one block
__global__ void k_data_norms(const double* c, const double* b, const double* h, int n, int p, int m,
                             IPMScalars* S) {
    __shared__ double sm[3 * 32];
    double a[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) a[0] = fmax(a[0], fabs(c[i]));
    for (int i = threadIdx.x; i < p; i += blockDim.x) a[1] = fmax(a[1], fabs(b[i]));
    for (int i = threadIdx.x; i < m; i += blockDim.x) a[2] = fmax(a[2], fabs(h[i]));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < 3; ++k) {
        a[k] = warp_max_nonneg(a[k]);
        if (lane == 0) sm[k * 32 + wid] = a[k];
    }
    __syncthreads();
    if (wid == 0) {
        for (int k = 0; k < 3; ++k) a[k] = warp_max_nonneg(lane < nw ? sm[k * 32 + lane] : 0.0);
        if (lane == 0) { S->c_inf = a[0]; S->b_inf = a[1]; S->h_inf = a[2]; }
    }
}

}  // namespace qoco

using namespace qoco;

struct qoco_gpu_cones {
    ConeView v;
    std::vector<void*> allocs;
    double* partial = nullptr;
};

// CUDA-event timing of the iteration's phases (enabled by qoco_gpu_set_profiling).
struct PhaseProfiler {
    bool on = false;
    bool factor_only = false;  // time the factorisation phase alone (two events per factorisation)
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec { int phase; cudaEvent_t a, b; int64_t launches; };
    std::vector<Rec> pending;
    qoco_gpu_profile tot;
    PhaseProfiler() { memset(&tot, 0, sizeof tot); }
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    // called after the stream was synchronised
    void flush() {
        for (const Rec& r : pending) {
            float ms = 0.0f;
            if (r.a && r.b && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                tot.ms[r.phase] += ms;
                tot.calls[r.phase] += 1;
                tot.launches[r.phase] += r.launches;
            }
        }
        pending.clear();
        used = 0;
    }
    ~PhaseProfiler() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

// Event pair timing one triangular solve on a factor with FP32 large fronts: the cost of a
// GMRES iteration, against which an FP64 refactor is weighed.
struct SolveTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    double ms = 0.0;  // the latest timed solve
    ~SolveTimer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

struct qoco_gpu_solver {
    qoco_gpu_settings st;
    SolveTimer stimer;
    PhaseProfiler prof;
    int64_t h2d_bytes = 0, d2h_bytes = 0;
    KKTPattern K;
    Symbolic S;
    int n = 0, m = 0, p = 0, N = 0;
    std::vector<void*> allocs;
    // device data
    int64_t* d_rowptr = nullptr;
    int* d_long_rows = nullptr;
    int* d_colidx = nullptr;
    double* d_val = nullptr;
    int64_t* d_w2slot = nullptr;
    int64_t* d_w2ptr = nullptr;
    double *d_c = nullptr, *d_b = nullptr, *d_h = nullptr;
    // iterate and work vectors
    double *xyz = nullptr, *s = nullptr, *d_aff = nullptr, *ds_aff = nullptr, *d_cmb = nullptr,
           *ds_cmb = nullptr;
    double *r = nullptr, *rhs = nullptr, *wbar = nullptr, *eta = nullptr, *lam = nullptr, *t = nullptr,
           *t1 = nullptr, *t2 = nullptr;
    double *sol_w = nullptr, *sol_xp = nullptr, *res = nullptr;
    double* partial = nullptr;
    int64_t partial_cap = 0;
    IPMScalars* d_S = nullptr;
    IPMScalars* h_S = nullptr;  // pinned
    KKTView kv;
    ConeView cv;
    FactorView fv;
    FactorPlan plan;
    int lpr = 4;
    bool have_factor = false;
    int64_t launches = 0;
    int refine_steps = 0;
    double last_berr = 0.0;
    // polls a device-side dependency wait may take before it gives up (each poll sleeps
    // ~32–64 ns): settings.wait_polls, or 20000000 (about a second)
    long long wait_polls = 20000000;
    bool have_solution = false;  // a solve completed (adjoint available)
    // CUDA graphs of the level-launch factorisation (per large-front precision) and of the
    // level-launch solves (per right-hand side / solution / accumulate triple); captured
    // on a private stream once, replayed on the caller's stream
    struct Graph { const void* r = nullptr; void* x = nullptr; int acc = 0; cudaGraphExec_t exec = nullptr; int launches = 0; };
    Graph fgraph[2];
    std::vector<Graph> sgraphs;
    Graph bgraph;
    cudaStream_t cap_stream = nullptr;
    // batch of independent instances (qoco_gpu_setup_batch)
    bool batch = false;
    BatchView bv;
    int batch_L = 0;                   // stacked orthant dimension
    double *b_items = nullptr, *b_shift = nullptr, *b_aux = nullptr;
    std::vector<int> h_xo, h_yo, h_lo, h_ko, h_so;
    // the persistent batched kernel (batch_schedule 0 or 6): its arguments, the tile
    // configuration picked at the first solve (warps per CTA, thread-front split, resident
    // warps per SM), the persistent grid per candidate and the captured launch graph
    bool fused = false;
    BatchIPMArgs bargs;
    int fused_nw = 0, fused_split = 0, fused_dense = 0;
    int fused_grid[6] = {0, 0, 0, 0, 0, 0};  // [warp-count index · 2 + dense]
    int fp32_factors = 0, fp64_escalations = 0;
    // mixed precision: FP32 large fronts allowed for this solve, and the number of
    // consecutive FP32 factorisations whose refinement failed (two stop the retries)
    bool mixed_ok = false;
    int fp32_fail_streak = 0;
    // smallest signed pivot accepted in a scaled FP32 front, raised tenfold (up to
    // kPiv32Max) after each breakdown of an FP32 factor within one solve
    double piv32 = 0.0;
    int fp32_floor_raises = 0;
    // GMRES refinement (mixed precision): basis V ((restart + 1) × N), work vector, zero
    // vector, Hessenberg column / coefficients (device), dot-product partials
    double *kv_basis = nullptr, *kv_z = nullptr, *kv_zero = nullptr, *kv_h = nullptr, *kv_y = nullptr,
           *kv_part = nullptr;
    // GMRES row scaling: den = |K||x| + |r| per row at the start of a cycle, and a work vector
    double *kv_den = nullptr, *kv_t = nullptr;
    int krylov_steps = 0;
    // adjoint: KKT position (row, column) of one slot of each data entry [P | A | G]
    int *d_adj_a = nullptr, *d_adj_b = nullptr;
    int adj_steps = 0, adj_refactored = 0;
    double adj_berr = 0.0;
    // parametric update: KKT slots fed by data and their source index in [P | A | G]
    int64_t *d_data_slot = nullptr, *d_data_src = nullptr;
    int64_t n_data_slot = 0;
    int solve_epoch = 0;   // flag value of the latest dataflow solve
    // the right-hand side whose forward sweep the latest dataflow factorisation ran (its
    // result is in sol_w, flagged with fused_epoch), until the next solve uses or drops it
    const double* fused_rhs = nullptr;
    int fused_epoch = 0;
    int factor_epoch = 0;  // flag value of the latest dataflow factorisation
    qoco_gpu_info info;
    std::string msg;
};

namespace {

template <class T>
int dalloc(qoco_gpu_solver* S, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    QOCO_CUDA_TRY(cudaMalloc((void**)p, count * sizeof(T)));
    S->allocs.push_back(*p);
    return 0;
}
template <class T>
int dcopy(qoco_gpu_solver* S, T** p, const std::vector<T>& v) {
    int rc = dalloc(S, p, v.size());
    if (rc) return rc;
    if (!v.empty()) QOCO_CUDA_TRY(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    S->h2d_bytes += (int64_t)(v.size() * sizeof(T));
    return 0;
}

// Pivot floor of the scaled FP32 large fronts: start of each solve, and the largest the
// breakdown retries raise it to (1e-5 → 1e-4 → 1e-3 → 1e-2) before refactoring in FP64.
constexpr double kPiv32Start = 1e-5, kPiv32Max = 1e-2;

int set_piv32(qoco_gpu_solver* S, double v, cudaStream_t st) {
    S->piv32 = v;
    QOCO_CUDA_TRY(cudaMemcpyAsync(const_cast<double*>(S->fv.piv32), &S->piv32, sizeof(double),
                                  cudaMemcpyHostToDevice, st));
    return 0;
}

// Records an event pair around one phase when profiling is on.
struct Phase {
    qoco_gpu_solver* S;
    int phase;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    int64_t l0;
    Phase(qoco_gpu_solver* s_, int ph, cudaStream_t st_) : S(s_), phase(ph), st(st_), l0(s_->launches) {
        if (S->prof.on && (!S->prof.factor_only || phase == QOCO_GPU_PHASE_FACTOR) && (a = S->prof.next()))
            cudaEventRecord(a, st);
    }
    ~Phase() {
        if (!a) return;
        cudaEvent_t b = S->prof.next();
        if (b) cudaEventRecord(b, st);
        S->prof.pending.push_back({phase, a, b, S->launches - l0});
    }
};

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

int grid(int n, int t = 256) { return (n + t - 1) / t; }

int build_cone_view(qoco_gpu_solver* S, const KKTPattern& K) {
    ConeView& c = S->cv;
    c.l = K.l;
    c.nsoc = K.nsoc;
    c.m = K.m;
    std::vector<int> off(K.nsoc), dim(K.nsoc), sm, lg;
    for (int k = 0; k < K.nsoc; ++k) {
        off[k] = K.cone_off[k];
        dim[k] = K.q[k];
        (K.q[k] <= kSmallCone ? sm : lg).push_back(k);
    }
    int* p;
    int rc;
    if ((rc = dcopy(S, &p, off))) return rc;
    c.off = p;
    if ((rc = dcopy(S, &p, dim))) return rc;
    c.dim = p;
    if ((rc = dcopy(S, &p, sm))) return rc;
    c.small = p;
    if ((rc = dcopy(S, &p, lg))) return rc;
    c.large = p;
    c.nsmall = (int)sm.size();
    c.nlarge = (int)lg.size();
    std::vector<int> wide;
    for (int k = 0; k < K.nsoc; ++k)
        if (K.q[k] > kWideCone) {
            wide.push_back(k);
            c.wide_maxd = std::max(c.wide_maxd, K.q[k]);
        }
    if (!wide.empty()) {
        if ((rc = dcopy(S, &p, wide))) return rc;
        c.wide = p;
        c.nwide = (int)wide.size();
    }
    return 0;
}

int upload(qoco_gpu_solver* S, const double* c, const double* b, const double* h) {
    if (S->st.wait_polls > 0) S->wait_polls = S->st.wait_polls;
    const KKTPattern& K = S->K;
    const Symbolic& Y = S->S;
    int rc;
    const int N = K.N, m = K.m;
    if ((rc = dcopy(S, &S->d_rowptr, K.rowptr))) return rc;
    if ((rc = dcopy(S, &S->d_colidx, K.colidx))) return rc;
    if ((rc = dcopy(S, &S->d_val, K.val0))) return rc;
    if ((rc = dcopy(S, &S->d_w2slot, K.w2_slot))) return rc;
    if ((rc = dcopy(S, &S->d_w2ptr, K.w2_ptr))) return rc;
    std::vector<double> vc(c, c + K.n), vb(K.p, 0.0), vh(K.m, 0.0);
    if (b) vb.assign(b, b + K.p);
    if (h) vh.assign(h, h + K.m);
    if ((rc = dcopy(S, &S->d_c, vc))) return rc;
    if ((rc = dcopy(S, &S->d_b, vb))) return rc;
    if ((rc = dcopy(S, &S->d_h, vh))) return rc;
    if ((rc = build_cone_view(S, K))) return rc;
    S->kv.N = N; S->kv.n = K.n; S->kv.p = K.p; S->kv.m = K.m;
    S->kv.rowptr = S->d_rowptr; S->kv.colidx = S->d_colidx; S->kv.val = S->d_val;
    std::vector<int> long_rows;
    int64_t long_nnz = 0;
    for (int i = 0; i < N; ++i)
        if (K.rowptr[i + 1] - K.rowptr[i] > kLongRow) {
            long_rows.push_back(i);
            long_nnz += K.rowptr[i + 1] - K.rowptr[i];
        }
    if (!long_rows.empty()) {
        if ((rc = dcopy(S, &S->d_long_rows, long_rows))) return rc;
        S->kv.long_rows = S->d_long_rows;
        S->kv.n_long = (int)long_rows.size();
    }
    const int n_short = N - (int)long_rows.size();
    const double avg = n_short ? (double)(K.nnz() - long_nnz) / n_short : 1.0;
    // lanes per KKT row in the row kernels: one thread per row for the very sparse rows
    // of stage-structured problems (no shuffles, one row-pointer load per row)
    S->lpr = avg <= 6 ? 1 : avg <= 12 ? 2 : avg <= 24 ? 4 : avg <= 48 ? 8 : avg <= 96 ? 16 : 32;

    // symbolic structure
    FactorView& f = S->fv;
    int* pi;
    int64_t* pl;
    std::vector<int> first(Y.sn_first.begin(), Y.sn_first.end() - 1);
    if ((rc = dcopy(S, &pi, first))) return rc; f.first = pi;
    if ((rc = dcopy(S, &pi, Y.sn_ncol))) return rc; f.ncol = pi;
    if ((rc = dcopy(S, &pi, Y.sn_nrow))) return rc; f.nrow = pi;
    if ((rc = dcopy(S, &pl, Y.row_ptr))) return rc; f.row_ptr = pl;
    if ((rc = dcopy(S, &pi, Y.rows))) return rc; f.rows = pi;
    if ((rc = dcopy(S, &pl, Y.front_off))) return rc; f.front_off = pl;
    if ((rc = dcopy(S, &pl, Y.upd_off))) return rc; f.upd_off = pl;
    if ((rc = dcopy(S, &pi, Y.rel))) return rc; f.rel = pi;
    if ((rc = dcopy(S, &pi, Y.child_ptr))) return rc; f.child_ptr = pi;
    if ((rc = dcopy(S, &pi, Y.child))) return rc; f.child = pi;
    {
        std::vector<ChildInfo> ci(Y.child.size());
        for (size_t k = 0; k < Y.child.size(); ++k) {
            const int ch = Y.child[k];
            const int fc = Y.sn_nrow[ch], cc = Y.sn_ncol[ch];
            ci[k].u_off = Y.front_off[ch] + (int64_t)cc * fc + cc;
            ci[k].rel_off = Y.upd_off[ch];
            ci[k].fc = fc;
            ci[k].r = fc - cc;
        }
        ChildInfo* pc;
        if ((rc = dcopy(S, &pc, ci))) return rc;
        f.cinfo = pc;
    }
    if ((rc = dcopy(S, &pl, Y.amap_ptr))) return rc; f.amap_ptr = pl;
    if ((rc = dcopy(S, &pl, Y.amap_slot))) return rc; f.amap_slot = pl;
    if ((rc = dcopy(S, &pl, Y.amap_off))) return rc; f.amap_off = pl;
    signed char* pc;
    if ((rc = dcopy(S, &pc, Y.dsign))) return rc; f.dsign = pc;
    if ((rc = dcopy(S, &pi, Y.perm))) return rc; f.perm = pi;
    if ((rc = dcopy(S, &pi, Y.sn_parent))) return rc; f.parent = pi;
    double* pd;
    if ((rc = dalloc(S, &pd, (size_t)Y.front_entries))) return rc; f.front = pd;
    if ((rc = dalloc(S, &pd, (size_t)Y.upd_off[Y.ns]))) return rc; f.upd = pd;
    if ((rc = dalloc(S, &pd, (size_t)N))) return rc; f.dinv = pd;
    if ((rc = dalloc(S, &pi, 1))) return rc; f.nreg = pi;
    f.eps = S->st.static_reg;
    f.eps32 = S->st.mixed_reg;
    f.dyn_thresh = S->st.dyn_reg_thresh;
    f.dyn_value = S->st.dyn_reg_value;

    // launch plan: subtree tasks + level lists
    PlanHost ph;
    build_plan(Y, &ph);
    {
        int max_small = 0, max_big = 0;
        std::vector<char> is_big(Y.ns, 0);
        for (int s : ph.big) is_big[s] = 1;
        for (int s = 0; s < Y.ns; ++s)
            (is_big[s] ? max_big : max_small) = std::max(is_big[s] ? max_big : max_small, Y.sn_nrow[s]);
        // large fronts index rows and columns with int and their entries with int64_t
        if (max_small > kMaxSolveFront || max_small > kMaxFactorFront || max_big > (1 << 24)) {
            S->msg = "a supernode front exceeds the factor/solve kernels' limits";
            return QOCO_GPU_ERR_NOT_IMPLEMENTED;
        }
    }
    FactorPlan& P = S->plan;
    P.levels = ph.levels;
    for (int s : ph.big) {
        P.big_s.push_back(s);
        P.big_f.push_back(Y.sn_nrow[s]);
        P.big_c.push_back(Y.sn_ncol[s]);
        P.big_front_off.push_back(Y.front_off[s]);
        P.big_amap_n.push_back(Y.amap_ptr[s + 1] - Y.amap_ptr[s]);
        P.max_big_f = std::max(P.max_big_f, Y.sn_nrow[s]);
    }
    if (P.max_big_f) {
        // leaf groups: childless children of a large front (c ≤ 8) sharing their update
        // rows, at least kMinGroup of them
        constexpr int kMinGroup = 32, kMaxLeafCols = 8;
        std::vector<signed char> skip(Y.ns, 0);
        int64_t max_rK = 0, max_tiles = 0, max_upd = 0;
        for (size_t idx = 0; idx < P.big_s.size(); ++idx) {
            const int s = P.big_s[idx];
            std::map<std::pair<int, uint64_t>, std::vector<int>> by_rows;
            for (int k = Y.child_ptr[s]; k < Y.child_ptr[s + 1]; ++k) {
                const int ch = Y.child[k];
                if (Y.child_ptr[ch + 1] > Y.child_ptr[ch]) continue;
                const int c = Y.sn_ncol[ch], r = Y.sn_nrow[ch] - c;
                if (c > kMaxLeafCols || r <= 0) continue;
                uint64_t hsh = 1469598103934665603ull;
                for (int i = 0; i < r; ++i) hsh = (hsh ^ (uint64_t)Y.rel[Y.upd_off[ch] + i]) * 1099511628211ull;
                by_rows[{r, hsh}].push_back(ch);
            }
            for (auto& kv : by_rows) {
                std::vector<int>& mem = kv.second;
                const int r = kv.first.first;
                // keep the members whose relative indices equal the first member's exactly
                const int* rel0 = &Y.rel[Y.upd_off[mem[0]]];
                std::vector<int> same;
                for (int ch : mem)
                    if (std::equal(rel0, rel0 + r, &Y.rel[Y.upd_off[ch]])) same.push_back(ch);
                if ((int)same.size() < kMinGroup) continue;
                FactorPlan::LeafGroup g;
                g.big_idx = (int)idx;
                g.r = r;
                g.nmem = (int)same.size();
                g.rel_off = Y.upd_off[same[0]];
                // member columns that reach the update rows: a member is a leaf, so its
                // columns' patterns are its KKT entries plus the fill among its own pivots
                std::vector<int> gmem, gloc;
                std::vector<unsigned char> pat;
                for (int w = 0; w < g.nmem; ++w) {
                    const int ch = same[w], f = Y.sn_nrow[ch], c = Y.sn_ncol[ch];
                    pat.assign((size_t)c * f, 0);
                    for (int64_t e = Y.amap_ptr[ch]; e < Y.amap_ptr[ch + 1]; ++e) pat[Y.amap_off[e]] = 1;
                    for (int t = 0; t < c; ++t)
                        for (int i = t + 1; i < c; ++i)
                            if (pat[(size_t)t * f + i])
                                for (int q2 = i + 1; q2 < f; ++q2) pat[(size_t)i * f + q2] |= pat[(size_t)t * f + q2];
                    for (int t = 0; t < c; ++t) {
                        bool border = false;
                        for (int q2 = c; q2 < f && !border; ++q2) border = pat[(size_t)t * f + q2] != 0;
                        if (border) { gmem.push_back(w); gloc.push_back(t); }
                    }
                    skip[ch] = 1;
                }
                g.K = (int)gmem.size();
                std::vector<int64_t> uo;
                for (int ch : same) uo.push_back(Y.upd_off[ch]);
                if ((rc = dcopy(S, &g.d_updoff, uo))) return rc;
                if ((rc = dcopy(S, &g.d_members, same))) return rc;
                if ((rc = dcopy(S, &g.d_gmem, gmem))) return rc;
                if ((rc = dcopy(S, &g.d_gloc, gloc))) return rc;
                max_rK = std::max(max_rK, (int64_t)r * g.K);
                max_upd = std::max(max_upd, (int64_t)((g.nmem + 255) / 256) * r);  // solve partials
                const int64_t nt = (r + kGroupTile - 1) / kGroupTile;
                max_tiles = std::max(max_tiles, nt * (nt + 1) / 2);
                P.groups.push_back(g);
            }
        }
        // row-ownership lists of the large fronts' children (extend-add and solve gather)
        std::vector<int64_t> ea_ptr;
        std::vector<int> ea_child, ea_pos;
        for (size_t idx = 0; idx < P.big_s.size(); ++idx) {
            const int s = P.big_s[idx], f = Y.sn_nrow[s];
            P.big_ea_off.push_back((int64_t)ea_ptr.size());
            std::vector<int64_t> cnt(f + 1, 0);
            for (int k = Y.child_ptr[s]; k < Y.child_ptr[s + 1]; ++k) {
                const int ch = Y.child[k], r = Y.sn_nrow[ch] - Y.sn_ncol[ch];
                if (skip[ch]) continue;  // a leaf-group member: reaches the parent through its group
                for (int jj = 0; jj < r; ++jj) cnt[Y.rel[Y.upd_off[ch] + jj] + 1]++;
            }
            for (int q = 0; q < f; ++q) cnt[q + 1] += cnt[q];
            const int64_t base = (int64_t)ea_child.size();
            for (int q = 0; q <= f; ++q) ea_ptr.push_back(base + cnt[q]);
            ea_child.resize(base + cnt[f]);
            ea_pos.resize(base + cnt[f]);
            std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
            for (int k = Y.child_ptr[s]; k < Y.child_ptr[s + 1]; ++k) {
                const int ch = Y.child[k], r = Y.sn_nrow[ch] - Y.sn_ncol[ch];
                if (skip[ch]) continue;
                for (int jj = 0; jj < r; ++jj) {
                    const int64_t e = base + fill[Y.rel[Y.upd_off[ch] + jj]]++;
                    ea_child[e] = k;
                    ea_pos[e] = jj;
                }
            }
        }
        if ((rc = dcopy(S, &P.d_ea_ptr, ea_ptr))) return rc;
        if (!P.groups.empty()) {
            P.grp_split = 128;
            if ((rc = dalloc(S, &P.grp_L, (size_t)max_rK))) return rc;
            if ((rc = dalloc(S, &P.grp_W, (size_t)max_rK))) return rc;
            if ((rc = dalloc(S, &P.grp_part,
                             (size_t)std::max<int64_t>(P.grp_split * max_tiles * kGroupTile * kGroupTile, max_upd))))
                return rc;
            signed char* pskip;
            if ((rc = dcopy(S, &pskip, skip))) return rc;
            S->fv.skip = pskip;
        }
        if (!ea_child.empty()) {
            if ((rc = dcopy(S, &P.d_ea_child, ea_child))) return rc;
            if ((rc = dcopy(S, &P.d_ea_pos, ea_pos))) return rc;
        }
        int64_t nlinv = 0;
        for (size_t idx = 0; idx < P.big_s.size(); ++idx) {
            P.big_linv_off.push_back(nlinv);
            nlinv += (int64_t)((P.big_c[idx] + kBigNB - 1) / kBigNB) * kBigNB * kBigNB;
        }
        if ((rc = dalloc(S, &P.big_linv, std::max<int64_t>(nlinv, 1)))) return rc;
        // panel rows W (and, for FP32 fronts, row-major L) of up to 4·kBigNB columns
        double* pw;
        if ((rc = dalloc(S, &pw, (size_t)P.max_big_f * 4 * kBigNB))) return rc;
        P.big_w = pw;
        if ((rc = dalloc(S, &P.big_v, P.max_big_f))) return rc;
        if ((rc = dalloc(S, &P.big_y, P.max_big_f))) return rc;
        if (S->st.mixed_precision) {
            if ((rc = dalloc(S, &P.big_work32, (size_t)P.max_big_f * P.max_big_f))) return rc;
            if ((rc = dalloc(S, &P.big_split, (size_t)4 * P.max_big_f * 4 * kBigNB))) return rc;
            if ((rc = dalloc(S, &P.big_scale, (size_t)P.max_big_f))) return rc;
            double* pv;
            if ((rc = dalloc(S, &pv, 1))) return rc;
            f.piv32 = pv;
            if ((rc = dalloc(S, &f.bad32, 1))) return rc;
            if ((rc = set_piv32(S, kPiv32Start, nullptr))) return rc;
            if ((rc = big_tma_setup(P))) return rc;
            const size_t R = kKrylovRestart;
            if ((rc = dalloc(S, &S->kv_basis, (R + 1) * (size_t)N))) return rc;
            if ((rc = dalloc(S, &S->kv_z, (size_t)N))) return rc;
            if ((rc = dalloc(S, &S->kv_den, (size_t)N))) return rc;
            if ((rc = dalloc(S, &S->kv_t, (size_t)N))) return rc;
            if ((rc = dalloc(S, &S->kv_zero, (size_t)N))) return rc;
            QOCO_CUDA_TRY(cudaMemset(S->kv_zero, 0, sizeof(double) * N));
            if ((rc = dalloc(S, &S->kv_h, 2 * (R + 2) + 1))) return rc;
            if ((rc = dalloc(S, &S->kv_y, R))) return rc;
            if ((rc = dalloc(S, &S->kv_part, (size_t)krylov_partials()))) return rc;
        }
        int64_t max_blk = 0;
        for (size_t idx = 0; idx < P.big_s.size(); ++idx)
            max_blk = std::max<int64_t>(max_blk, (P.big_c[idx] + kBigNB - 1) / kBigNB);
        if ((rc = dalloc(S, &P.big_ctl, (size_t)(1 + max_blk)))) return rc;
        if ((rc = big_set_attributes())) return rc;
    }
    S->info.large_fronts = (int)ph.big.size();
    if ((rc = dcopy(S, &P.d_thread, ph.thread))) return rc;
    if ((rc = dcopy(S, &P.d_warp, ph.warp))) return rc;
    if ((rc = dcopy(S, &P.d_small, ph.small))) return rc;
    if ((rc = dcopy(S, &P.d_large, ph.large))) return rc;
    if ((rc = dcopy(S, &P.d_cta, ph.cta))) return rc;
    if ((rc = dcopy(S, &P.d_sthread, ph.sthread))) return rc;
    if ((rc = dcopy(S, &P.d_swarp, ph.swarp))) return rc;
    {
        int mwf = 0;
        for (const LevelPlan& L : ph.levels) mwf = std::max(mwf, L.max_swarp_f);
        P.nitems = (int)ph.items.size();
        if ((rc = dcopy(S, &P.d_items, ph.items))) return rc;
        if ((rc = dcopy(S, &P.d_tb_ptr, ph.tb_ptr))) return rc;
        std::vector<int> zeros(Y.ns, 0);
        if ((rc = dcopy(S, &P.d_fdone, zeros))) return rc;
        if ((rc = dcopy(S, &P.d_bdone, zeros))) return rc;
        const bool any_cta = !ph.cta.empty() || !ph.big.empty();
        if ((rc = plan_dataflow_solve(P, mwf, any_cta))) return rc;
        P.nfitems = (int)ph.fitems.size();
        if ((rc = dcopy(S, &P.d_fitems, ph.fitems))) return rc;
        if ((rc = dcopy(S, &P.d_ftb_ptr, ph.ftb_ptr))) return rc;
        if ((rc = dcopy(S, &P.d_fwg_ptr, ph.fwg_ptr))) return rc;
        if ((rc = dcopy(S, &P.d_cdone, zeros))) return rc;
        if ((rc = plan_dataflow_factor(P, ph.max_f, !ph.large.empty() || !ph.big.empty()))) return rc;
    }

    // data-entry maps (adjoint coordinates, parametric-update scatter list)
    {
        const int64_t nd = K.nnzP + K.nnzA + K.nnzG;
        std::vector<int> ca(nd, -1), cb(nd, -1);
        std::vector<int64_t> dslot, dsrc;
        dslot.reserve(2 * nd);
        dsrc.reserve(2 * nd);
        for (int i = 0; i < N; ++i)
            for (int64_t t = K.rowptr[i]; t < K.rowptr[i + 1]; ++t) {
                const int64_t k = K.src[t];
                if (k < 0) continue;
                if (ca[k] < 0) { ca[k] = i; cb[k] = K.colidx[t]; }
                dslot.push_back(t);
                dsrc.push_back(k);
            }
        if ((rc = dcopy(S, &S->d_adj_a, ca))) return rc;
        if ((rc = dcopy(S, &S->d_adj_b, cb))) return rc;
        if ((rc = dcopy(S, &S->d_data_slot, dslot))) return rc;
        if ((rc = dcopy(S, &S->d_data_src, dsrc))) return rc;
        S->n_data_slot = (int64_t)dslot.size();
    }

    // iterate / work vectors
    double** vecN[] = {&S->xyz, &S->d_aff, &S->d_cmb, &S->r, &S->rhs, &S->sol_w, &S->sol_xp, &S->res};
    for (double** v : vecN) if ((rc = dalloc(S, v, N))) return rc;
    double** vecM[] = {&S->s, &S->ds_aff, &S->ds_cmb, &S->wbar, &S->lam, &S->t, &S->t1, &S->t2};
    for (double** v : vecM) if ((rc = dalloc(S, v, m))) return rc;
    if ((rc = dalloc(S, &S->eta, K.nsoc))) return rc;
    const int np = std::max(row_partials(N, S->kv.n_long), 2 * std::max(1, max_step_partials(S->cv)));
    if ((rc = dalloc(S, &S->partial, np))) return rc;
    S->partial_cap = np;
    if ((rc = dalloc(S, &S->d_S, 1))) return rc;
    S->plan.df_err = &S->d_S->bar_err;
    S->plan.df_spins = S->wait_polls;
    QOCO_CUDA_TRY(cudaMallocHost((void**)&S->h_S, sizeof(IPMScalars)));

    IPMScalars hs;
    memset(&hs, 0, sizeof hs);
    auto inf = [](const double* v, int len) {
        double a = 0.0;
        for (int i = 0; i < len; ++i) a = std::max(a, std::fabs(v[i]));
        return a;
    };
    hs.c_inf = inf(vc.data(), K.n);
    hs.b_inf = inf(vb.data(), K.p);
    hs.h_inf = inf(vh.data(), K.m);
    hs.nu = K.l + K.nsoc;
    hs.abstol = S->st.abstol; hs.reltol = S->st.reltol;
    hs.abstol_inacc = S->st.abstol_inacc; hs.reltol_inacc = S->st.reltol_inacc;
    hs.refine_tol = S->st.refine_tol;
    hs.step_fraction = S->st.step_fraction;
    QOCO_CUDA_TRY(cudaMemcpy(S->d_S, &hs, sizeof hs, cudaMemcpyHostToDevice));
    return factor_set_attributes();
}

// ---- steps of the iteration ----------------------------------------------------
int sync_scalars(qoco_gpu_solver* S, cudaStream_t st) {
    QOCO_CUDA_TRY(cudaMemcpyAsync(S->h_S, S->d_S, sizeof(IPMScalars), cudaMemcpyDeviceToHost, st));
    QOCO_CUDA_TRY(cudaStreamSynchronize(st));
    S->d2h_bytes += (int64_t)sizeof(IPMScalars);
    if (S->prof.on) S->prof.flush();
    return 0;
}

// Captures `launch` (which returns its kernel count) into a graph on the private
// capture stream and instantiates it.
template <class F>
int capture_graph(qoco_gpu_solver* S, qoco_gpu_solver::Graph* g, F launch) {
    if (!S->cap_stream) QOCO_CUDA_TRY(cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    QOCO_CUDA_TRY(cudaStreamBeginCapture(S->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int n = launch(S->cap_stream);
    const cudaError_t e = cudaStreamEndCapture(S->cap_stream, &graph);
    if (e != cudaSuccess || n < 0) {
        if (graph) cudaGraphDestroy(graph);
        return n < 0 ? n : cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    }
    const cudaError_t e2 = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaGraphInstantiate", __FILE__, __LINE__);
    g->launches = n;
    return 0;
}

// Batch schedules: 1–4 are the per-instance kernels (launch_inst_factor), 5 the shared
// kernels every problem uses (dataflow launches, or level launches from graphs).
constexpr int kSharedSchedule = 5;

int factor_shared(qoco_gpu_solver* S, cudaStream_t st, const double* fwd_rhs) {
    S->fused_rhs = nullptr;
    if (S->plan.fdataflow) {
        DataflowState ds;
        ds.next = &S->d_S->sched_next;
        ds.err = &S->d_S->bar_err;
        ds.epoch = ++S->factor_epoch;
        ds.max_spins = S->wait_polls;
        FwdFuse fz;
        if (fwd_rhs && S->plan.dataflow) {  // the forward sweep of fwd_rhs in the same launch
            fz.rhs = fwd_rhs;
            fz.w = S->sol_w;
            fz.fdone = S->plan.d_fdone;
            fz.epoch = ++S->solve_epoch;
        }
        const int rc = launch_factor_dataflow(S->plan, S->fv, S->d_val, ds, st, fz);
        S->fused_rhs = fz.rhs;
        S->fused_epoch = fz.epoch;
        if (rc < 0) return rc;
        S->launches += rc;
        return 0;
    }
    // the level launches (and large-front kernel sequences) are the same every time:
    // replayed from a graph
    qoco_gpu_solver::Graph& g = S->fgraph[S->plan.big_fp32 ? 1 : 0];
    if (!g.exec) {
        const int rc = capture_graph(S, &g, [&](cudaStream_t cs) { return launch_factor(S->plan, S->fv, S->d_val, cs); });
        if (rc) return rc;
    }
    QOCO_CUDA_TRY(cudaGraphLaunch(g.exec, st));
    S->launches += g.launches;
    return 0;
}

int solve_shared(qoco_gpu_solver* S, const double* r, double* x, bool acc, cudaStream_t st) {
    const bool fused = S->fused_rhs && S->fused_rhs == r && !acc;
    S->fused_rhs = nullptr;
    if (S->plan.dataflow) {
        DataflowState ds;
        ds.next = &S->d_S->sched_next;
        ds.err = &S->d_S->bar_err;
        ds.epoch = fused ? S->fused_epoch : ++S->solve_epoch;
        ds.max_spins = S->wait_polls;
        const int rc = launch_solve_dataflow(S->plan, S->fv, r, S->sol_w, S->sol_xp, x, acc, ds, st, fused);
        if (rc < 0) return rc;
        S->launches += rc;
    } else {
        // level launches: one graph per (r, x, acc) triple (a handful per solver)
        qoco_gpu_solver::Graph* g = nullptr;
        for (auto& c : S->sgraphs)
            if (c.r == r && c.x == x && c.acc == (acc ? 1 : 0)) g = &c;
        if (!g) {
            qoco_gpu_solver::Graph ng;
            ng.r = r;
            ng.x = x;
            ng.acc = acc ? 1 : 0;
            const int rc = capture_graph(S, &ng, [&](cudaStream_t cs) {
                return launch_solve(S->plan, S->fv, r, S->sol_w, S->sol_xp, x, acc, cs);
            });
            if (rc) return rc;
            S->sgraphs.push_back(ng);
            g = &S->sgraphs.back();
        }
        QOCO_CUDA_TRY(cudaGraphLaunch(g->exec, st));
        S->launches += g->launches;
    }
    return 0;
}

int factor_with(qoco_gpu_solver* S, int v, cudaStream_t st, const double* fwd_rhs) {
    if (v >= 1 && v <= 4) {
        S->fused_rhs = nullptr;
        const int rc = launch_inst_factor(S->plan, S->fv, S->d_val, v, st);
        if (rc < 0) return rc;
        S->launches += rc;
        return 0;
    }
    return factor_shared(S, st, fwd_rhs);
}

int solve_with(qoco_gpu_solver* S, int v, const double* r, double* x, bool acc, cudaStream_t st) {
    if (v >= 1 && v <= 4) {
        S->fused_rhs = nullptr;
        const int rc = launch_inst_solve(S->plan, S->fv, r, S->sol_w, S->sol_xp, x, acc, v, st);
        if (rc < 0) return rc;
        S->launches += rc;
        return 0;
    }
    return solve_shared(S, r, x, acc, st);
}

// fwd_rhs: a right-hand side whose forward sweep the factorisation may run on the way
// (the next solve of fwd_rhs then runs only the backward sweep)
int factor_now(qoco_gpu_solver* S, cudaStream_t st, const double* fwd_rhs = nullptr) {
    {
        Phase ph(S, QOCO_GPU_PHASE_ROW, st);
        const int nl = launch_norm_inf(S->kv, S->lpr, S->partial, S->partial_cap, S->d_S, st);
        if (nl < 0) return QOCO_GPU_ERR_INVALID_ARG;
        S->launches += nl;
    }
    {
        Phase ph(S, QOCO_GPU_PHASE_FACTOR, st);
        const int rc = factor_with(S, S->plan.inst ? S->plan.inst_variant : kSharedSchedule, st, fwd_rhs);
        if (rc) return rc;
    }
    QOCO_CUDA_TRY(cudaGetLastError());
    if (S->plan.big_fp32) ++S->fp32_factors;
    S->have_factor = true;
    return 0;
}

int tri_solve(qoco_gpu_solver* S, const double* r, double* x, bool acc, cudaStream_t st) {
    Phase ph(S, QOCO_GPU_PHASE_SOLVE, st);
    return solve_with(S, S->plan.inst ? S->plan.inst_variant : kSharedSchedule, r, x, acc, st);
}

int refine_residual(qoco_gpu_solver* S, const double* x, const double* r, double* res, cudaStream_t st,
                    double* den = nullptr) {
    Phase ph(S, QOCO_GPU_PHASE_ROW, st);
    const int nl = launch_spmv_res(S->kv, S->lpr, x, r, res, S->partial, S->partial_cap, S->d_S, st,
                                   S->plan.big_fp32 || den, den);
    if (nl < 0) return QOCO_GPU_ERR_INVALID_ARG;
    S->launches += nl;
    return 0;
}

// Acceptance of a refined solve: the normwise backward error ‖r − Kx‖∞ / (‖K‖∞‖x‖∞ +
// ‖r‖∞) at refine_tol; on a factor with FP32 large fronts also the componentwise one,
// max_i |r − Kx|_i / (|K||x| + |r|)_i, at refine_tol.  Near the end of a solve ‖K‖∞ is
// ~1e16 (the −W² entries of inactive constraints), and a solve from an FP32 factor that
// met the normwise target alone could still be wrong in the rows of small scale (the
// equality rows), which stalled the interior-point iteration; an FP64 factor meets both
// by far.
bool solve_accepted(const qoco_gpu_solver* S) {
    const IPMScalars& h = *S->h_S;
    if (!h.refine_done || !std::isfinite(h.berr)) return false;
    return !S->plan.big_fp32 || h.berr_cw <= S->st.refine_tol;
}
// progress measure of the refinement (≤ 1: accepted, up to the refine_done flag)
double refine_error(const qoco_gpu_solver* S) {
    const IPMScalars& h = *S->h_S;
    const double e = h.berr / S->st.refine_tol;
    return S->plan.big_fp32 ? std::fmax(e, h.berr_cw / S->st.refine_tol) : e;
}

// GMRES refinement (GMRES-IR, Carson & Higham 2017–2018) on K x = r, K the unregularised
// KKT matrix (FP64 products), preconditioned by the current factor M (FP32 large fronts)
// and row-scaled: with D = diag(1/(|K||x| + |r|)) fixed at the start of a cycle, GMRES runs
// on D·K·M⁻¹·D⁻¹ (≈ I) from the scaled residual D(r − Kx), so that it minimises
// ‖D(r − Kx)‖₂, a bound on the componentwise backward error (and, since every row's
// denominator is at most ‖K‖∞‖x‖∞ + ‖r‖∞, on the normwise one).  The Krylov basis is
// orthogonalised by classical Gram–Schmidt applied twice, the least-squares problem
// reduced by Givens rotations on the host, and x += M⁻¹·D⁻¹·V·y at the end of a cycle;
// each cycle ends early when the GMRES residual estimate is below half the target, and
// is followed by the true residual.  Sets *ok when the solve is accepted.
// GMRES iterations worth spending before an FP64 refactor is cheaper: a GMRES iteration
// costs about 1.25 triangular solves (the timed one), an FP64 refactor its algorithmic
// flops at ~1 TFLOP/s (this part's FP64 rate); between 10 and 3 cycles of kKrylovRestart.
int gmres_budget(const qoco_gpu_solver* S) {
    const double fp64_ms = S->S.flops / 1e9;
    const double per = std::max(1.25 * S->stimer.ms, 1e-3);
    return (int)std::min(3.0 * kKrylovRestart, std::max(10.0, fp64_ms / per));
}

int gmres_refine(qoco_gpu_solver* S, const double* r, double* x, cudaStream_t st, bool* ok) {
    constexpr int R = kKrylovRestart, kCycles = 3;
    const int budget = gmres_budget(S);
    int used = 0;
    const int64_t N = S->N, ld = N;
    double* V = S->kv_basis;
    double* hd = S->kv_h;  // [0, R+2): first pass, [R+2, 2R+4): second pass, [2R+4]: ‖w‖²
    double* den = S->kv_den;
    *ok = false;
    std::vector<double> H((size_t)(R + 1) * R, 0.0), cs(R), sn(R), g(R + 1), hc(2 * (R + 2) + 1), y(R);
    int rc;
    for (int cycle = 0; cycle < kCycles && used < budget; ++cycle) {
        if ((rc = refine_residual(S, x, r, S->res, st, den))) return rc;
        // β = ‖D(r − Kx)‖₂, v_0 = D(r − Kx)/β
        S->launches += launch_row_scale(S->res, den, S->res, N, false, st);
        S->launches += launch_dots(S->res, ld, 1, S->res, N, S->kv_part, hd, false, st);
        S->launches += launch_scale_by_norm(S->res, V, N, hd, 1.0, st);
        QOCO_CUDA_TRY(cudaMemcpyAsync(S->h_S, S->d_S, sizeof(IPMScalars), cudaMemcpyDeviceToHost, st));
        QOCO_CUDA_TRY(cudaMemcpyAsync(hc.data(), hd, sizeof(double), cudaMemcpyDeviceToHost, st));
        QOCO_CUDA_TRY(cudaStreamSynchronize(st));
        if (S->prof.on) S->prof.flush();
        if (S->h_S->bar_err) return QOCO_GPU_ERR_DEVICE_TIMEOUT;
        if (!std::isfinite(S->h_S->berr)) return 0;
        if (solve_accepted(S)) { *ok = true; return 0; }
        const double beta = std::sqrt(hc[0]);
        const double target = 0.5 * S->st.refine_tol;
        if (!(beta > 0.0)) return 0;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < R; ++j) {
            double* vj = V + (int64_t)j * ld;
            double* w = V + (int64_t)(j + 1) * ld;
            S->launches += launch_row_scale(vj, den, S->kv_t, N, true, st);             // D⁻¹ v_j
            if ((rc = tri_solve(S, S->kv_t, S->kv_z, false, st))) return rc;           // z = M⁻¹ D⁻¹ v_j
            if ((rc = refine_residual(S, S->kv_z, S->kv_zero, w, st))) return rc;      // w = −K z
            S->launches += launch_row_scale(w, den, w, N, false, st);                   // w = −D K z
            // two classical Gram–Schmidt passes on the negated vector, then its norm
            S->launches += launch_dots(V, ld, j + 1, w, N, S->kv_part, hd, false, st);
            S->launches += launch_sub_combination(V, ld, j + 1, hd, w, N, st);
            S->launches += launch_dots(V, ld, j + 1, w, N, S->kv_part, hd + R + 2, false, st);
            S->launches += launch_sub_combination(V, ld, j + 1, hd + R + 2, w, N, st);
            S->launches += launch_dots(w, ld, 1, w, N, S->kv_part, hd + 2 * (R + 2), false, st);
            S->launches += launch_scale_by_norm(w, w, N, hd + 2 * (R + 2), -1.0, st);
            QOCO_CUDA_TRY(cudaMemcpyAsync(hc.data(), hd, sizeof(double) * hc.size(), cudaMemcpyDeviceToHost, st));
            QOCO_CUDA_TRY(cudaStreamSynchronize(st));
            S->d2h_bytes += (int64_t)(sizeof(double) * hc.size());
            if (S->prof.on) S->prof.flush();
            ++S->krylov_steps;
            ++used;
            double* h = &H[(size_t)j * (R + 1)];  // column j of the Hessenberg matrix
            for (int i = 0; i <= j; ++i) h[i] = -(hc[i] + hc[R + 2 + i]);
            h[j + 1] = std::sqrt(hc[2 * (R + 2)]);
            if (!std::isfinite(h[j + 1])) return 0;
            for (int i = 0; i < j; ++i) {  // earlier rotations
                const double a = cs[i] * h[i] + sn[i] * h[i + 1];
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
                h[i] = a;
            }
            const double rr = std::hypot(h[j], h[j + 1]);
            cs[j] = rr > 0.0 ? h[j] / rr : 1.0;
            sn[j] = rr > 0.0 ? h[j + 1] / rr : 0.0;
            h[j] = rr;
            h[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            if (std::fabs(g[j + 1]) <= target || !(hc[2 * (R + 2)] > 0.0) || used >= budget) break;
        }
        // y = R⁻¹ g, x += M⁻¹ D⁻¹ V y
        for (int i = k - 1; i >= 0; --i) {
            double a = g[i];
            for (int c = i + 1; c < k; ++c) a -= H[(size_t)c * (R + 1) + i] * y[c];
            y[i] = a / H[(size_t)i * (R + 1) + i];
        }
        QOCO_CUDA_TRY(cudaMemcpyAsync(S->kv_y, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        S->launches += launch_combination(V, ld, k, S->kv_y, S->kv_z, N, st);
        S->launches += launch_row_scale(S->kv_z, den, S->kv_t, N, true, st);
        if ((rc = tri_solve(S, S->kv_t, x, true, st))) return rc;
    }
    if ((rc = refine_residual(S, x, r, S->res, st))) return rc;
    if ((rc = sync_scalars(S, st))) return rc;
    if (S->h_S->bar_err) return QOCO_GPU_ERR_DEVICE_TIMEOUT;
    *ok = solve_accepted(S);
    return 0;
}

// x = K_ε⁻¹ r refined against K until the backward error target (r, x device, N).  On a
// factor with FP32 large fronts, a plain refinement that stalls (the backward error not
// halving in a step) or misses the target goes on with GMRES refinement; if that misses
// too, the solve refactors in FP64 (for the rest of the current solve) and starts over.
int solve_refine(qoco_gpu_solver* S, const double* r, double* x, cudaStream_t st) {
    for (;;) {
        if (S->plan.big_fp32 && !S->stimer.a && cudaEventCreate(&S->stimer.a) == cudaSuccess)
            if (cudaEventCreate(&S->stimer.b) != cudaSuccess) S->stimer.b = nullptr;
        const bool timed = S->plan.big_fp32 && S->stimer.a && S->stimer.b;
        if (timed) QOCO_CUDA_TRY(cudaEventRecord(S->stimer.a, st));
        int rc0 = tri_solve(S, r, x, false, st);
        if (rc0) return rc0;
        if (timed) QOCO_CUDA_TRY(cudaEventRecord(S->stimer.b, st));
        int steps = 0;
        double prev = INFINITY;
        for (;;) {
            int rc = refine_residual(S, x, r, S->res, st);
            if (rc) return rc;
            QOCO_CUDA_TRY(cudaGetLastError());
            if ((rc = sync_scalars(S, st))) return rc;
            if (S->h_S->bar_err) return QOCO_GPU_ERR_DEVICE_TIMEOUT;
            if (timed && steps == 0) {
                float ms = 0.0f;
                if (cudaEventElapsedTime(&ms, S->stimer.a, S->stimer.b) == cudaSuccess) S->stimer.ms = ms;
            }
            if (solve_accepted(S) || steps >= S->st.max_refine) break;
            const double err = refine_error(S);
            // an FP32 factor whose refinement no longer halves the error: GMRES takes over
            if (S->plan.big_fp32 && S->kv_basis && steps >= 2 && !(err < 0.5 * prev)) break;
            prev = err;
            if ((rc = tri_solve(S, S->res, x, true, st))) return rc;
            ++steps;
        }
        S->refine_steps += steps;
        S->last_berr = S->h_S->berr;
        bool ok = solve_accepted(S);
        if (ok && S->plan.big_fp32) S->fp32_fail_streak = 0;
        if (S->st.verbose >= 2)
            printf("     refine: %d steps, backward error %.3e, componentwise %.3e (%s factor)%s\n", steps,
                   S->h_S->berr, S->h_S->berr_cw, S->plan.big_fp32 ? "FP32 large fronts" : "FP64",
                   ok ? "" : " - target missed");
        if (!ok && S->plan.big_fp32) {
            // a factor that broke down (a non-finite or overgrown entry in a scaled FP32
            // front): FP32 again with a ten times larger pivot floor while it is below
            // kPiv32Max, else FP64
            int bad = 0;
            QOCO_CUDA_TRY(cudaMemcpyAsync(&bad, S->fv.bad32, sizeof(int), cudaMemcpyDeviceToHost, st));
            QOCO_CUDA_TRY(cudaStreamSynchronize(st));
            S->d2h_bytes += (int64_t)sizeof(int);
            if (bad && S->piv32 < 0.5 * kPiv32Max) {
                int rc = set_piv32(S, 10.0 * S->piv32, st);
                if (rc) return rc;
                ++S->fp32_floor_raises;
                if (S->st.verbose >= 2)
                    printf("     FP32 factor broke down: refactoring with pivot floor %.0e\n", S->piv32);
                if ((rc = factor_now(S, st))) return rc;
                continue;
            }
            if (bad) S->h_S->berr = INFINITY;  // no GMRES on a broken factor
        }
        if (!ok && S->plan.big_fp32 && S->kv_basis && std::isfinite(S->h_S->berr)) {
            const int k0 = S->krylov_steps;
            int rc = gmres_refine(S, r, x, st, &ok);
            if (rc) return rc;
            S->last_berr = S->h_S->berr;
            if (S->st.verbose >= 2)
                printf("     GMRES: %d iterations, backward error %.3e, componentwise %.3e%s\n",
                       S->krylov_steps - k0, S->h_S->berr, S->h_S->berr_cw,
                       ok ? "" : " - target missed, refactoring in FP64");
            if (ok) S->fp32_fail_streak = 0;
        }
        if (ok || !S->plan.big_fp32) return 0;
        S->plan.big_fp32 = false;
        ++S->fp32_fail_streak;
        ++S->fp64_escalations;
        int rc = factor_now(S, st);
        if (rc) return rc;
    }
}

int cone_launch_count(const ConeView& c) { return cone_grid(c).blocks() ? 1 : 0; }

int reset_barrier(qoco_gpu_solver* S, cudaStream_t st) {
    QOCO_CUDA_TRY(cudaMemsetAsync(&S->d_S->bar_count, 0, 4 * sizeof(unsigned int), st));
    return 0;
}

int fused_grid_index(int nw, int dense) { return 2 * (nw == 1 ? 0 : nw == 2 ? 1 : 2) + dense; }

// the batched kernel with tile configuration (nw, split, dense) over the first nb instances
// of the queue (all of them for a solve, a sample when tuning)
int launch_fused(qoco_gpu_solver* S, int nw, int split, int dense, int nb, cudaStream_t st) {
    BatchIPMArgs A = S->bargs;
    const FactorPlan::InstSched& I = S->plan.isched[split ? 0 : 1];
    A.lv_ptr = I.d_lv_ptr;
    A.ent = I.d_ent;
    A.sched = I.d_sched;
    A.B.nb = nb;
    const int grid = std::min(nb, S->fused_grid[fused_grid_index(nw, dense)]);
    return launch_batch_ipm(A, nw, dense, grid, st);
}

// Tile configuration of the batched kernel: warps per CTA (1, 2, 4; more warps share an
// instance's levels, fewer let more instances run side by side) × 16 or 32 resident warps
// per SM (128 or 64 registers per thread), fronts of order ≤ 8 one per thread.  Each
// candidate solves the whole batch once, after one untimed launch over one instance per
// CTA that takes the first-launch costs; a sample would mislead: the steady state of the
// persistent queue needs several instances per CTA, and the largest grids hold ~2400 CTAs.
// The search assumes the time is unimodal in the warps per CTA: from 4 warps (16 per SM)
// it halves the warps while that pays, then times the other residency of the best width
// (MPC batch of 4096: 3 of the 6 launches; the six times were 65, 69, 71, 74, 93, 99 ms).
int tune_fused(qoco_gpu_solver* S, cudaStream_t st) {
    cudaEvent_t e0, e1;
    QOCO_CUDA_TRY(cudaEventCreate(&e0));
    QOCO_CUDA_TRY(cudaEventCreate(&e1));
    const int nb = S->bv.nb, split = 1;
    float best = 0.0f;
    int rc = 0;
    bool warm = false;
    // times candidate (nw, dense); false when it is not available or the launch failed
    auto trial = [&](int nw, int dense, float* ms) -> bool {
        *ms = 0.0f;
        if (rc || !S->fused_grid[fused_grid_index(nw, dense)]) return false;
        if (!warm) {
            const int nl = launch_fused(S, nw, split, dense, std::min(nb, S->fused_grid[fused_grid_index(nw, dense)]), st);
            if (nl < 0) { rc = nl; return false; }
            warm = true;
        }
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = QOCO_GPU_ERR_CUDA; return false; }
        const int nl = launch_fused(S, nw, split, dense, nb, st);
        if (nl < 0) { rc = nl; return false; }
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = QOCO_GPU_ERR_CUDA;
            return false;
        }
        cudaEventElapsedTime(ms, e0, e1);
        if (S->st.verbose >= 2)
            printf("     batch tile: %d warps per CTA, %d warps per SM: %.3f ms\n", nw, dense ? 32 : 16, *ms);
        if (!S->fused_nw || *ms < best) {
            best = *ms;
            S->fused_nw = nw;
            S->fused_split = split;
            S->fused_dense = dense;
        }
        return true;
    };
    float ms = 0.0f;
    for (int nw = 4; nw >= 1 && !rc; nw /= 2) {
        const int before = S->fused_nw;
        if (!trial(nw, 0, &ms) && !rc && !trial(nw, 1, &ms)) continue;  // width unavailable: try the next
        if (before && S->fused_nw == before) break;                      // halving did not pay
    }
    if (!rc && S->fused_nw) trial(S->fused_nw, 1 - S->fused_dense, &ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    QOCO_CUDA_TRY(cudaGetLastError());
    return S->fused_nw ? 0 : QOCO_GPU_ERR_CUDA;
}

// One batched solve: the persistent kernel, the per-batch summary and its read-back,
// replayed from a CUDA graph captured at the first solve (after the tuning).
int run_fused(qoco_gpu_solver* S, cudaStream_t st) {
    int rc;
    if (!S->fused_nw && (rc = tune_fused(S, st))) return rc;
    if (!S->bgraph.exec) {
        rc = capture_graph(S, &S->bgraph, [&](cudaStream_t cs) {
            const int nl = launch_fused(S, S->fused_nw, S->fused_split, S->fused_dense, S->bv.nb, cs);
            if (nl < 0) return nl;
            launch_batch_summary(S->bv, S->d_S, cs);
            if (cudaMemcpyAsync(S->h_S, S->d_S, sizeof(IPMScalars), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
                return (int)QOCO_GPU_ERR_CUDA;
            return nl + 1;
        });
        if (rc) return rc;
    }
    QOCO_CUDA_TRY(cudaGraphLaunch(S->bgraph.exec, st));
    QOCO_CUDA_TRY(cudaStreamSynchronize(st));
    S->launches += S->bgraph.launches;
    S->d2h_bytes += (int64_t)sizeof(IPMScalars);
    const IPMScalars& h = *S->h_S;
    S->info.iters = h.max_iters;
    S->info.gap = h.gap;
    S->info.pobj = S->info.dobj = S->info.pres = S->info.dres = 0.0;
    S->info.batch_schedule_used = 6;
    if (h.nonfinite) return QOCO_GPU_ERR_NUMERICAL;
    if (h.converged) return QOCO_GPU_SOLVED;
    return h.converged_inacc ? QOCO_GPU_SOLVED_INACCURATE : QOCO_GPU_MAX_ITER;
}

int run_solve(qoco_gpu_solver* S, cudaStream_t st) {
    if (S->batch && S->fused) return run_fused(S, st);
    const int n = S->n, p = S->p, m = S->m, N = S->N;
    const ConeView& cv = S->cv;
    const int cl = cone_launch_count(cv);
    int rc;
    S->refine_steps = 0;
    S->fp32_factors = 0;
    S->fp64_escalations = 0;
    S->krylov_steps = 0;
    S->mixed_ok = S->st.mixed_precision != 0 && S->plan.max_big_f > 0 && S->plan.big_work32;
    S->fp32_fail_streak = 0;
    S->fp32_floor_raises = 0;
    S->plan.big_fp32 = S->mixed_ok;
    if (S->mixed_ok && (rc = set_piv32(S, kPiv32Start, st))) return rc;
    if ((rc = reset_barrier(S, st))) return rc;
    // initial point: K(W = I) [x; y; z] = [−c; b; h], s = −z, shift s and z into the cone
    S->launches += launch_w2_identity(cv, S->d_val, S->d_w2slot, S->d_w2ptr, st);
    k_init_rhs<<<grid(N), 256, 0, st>>>(S->rhs, S->d_c, S->d_b, S->d_h, n, p, m);
    S->launches += 1;
    if ((rc = factor_now(S, st, S->rhs))) return rc;
    if ((rc = solve_refine(S, S->rhs, S->d_cmb, st))) return rc;
    k_init_iterate<<<grid(N), 256, 0, st>>>(S->d_cmb, S->xyz, S->s, n, p, m);
    S->launches += 1;
    double* z = S->xyz + n + p;
    const bool B = S->batch;
    if (B) {
        // per-instance iteration counts and convergence flags start over
        QOCO_CUDA_TRY(cudaMemsetAsync(S->bv.conv, 0, sizeof(int) * S->bv.nb, st));
        QOCO_CUDA_TRY(cudaMemsetAsync(S->bv.iters, 0xff, sizeof(int) * S->bv.nb, st));
    }
    if (B && m > 0) {
        S->launches += launch_batch_shift(cv, S->bv, S->s, z, S->b_items, S->b_shift, st);
    } else if (m > 0) {
        launch_shift_measure(cv, S->s, z, S->partial, st);
        k_shift_finalize<<<1, 256, 0, st>>>(S->partial, max_step_partials(cv), S->d_S);
        launch_shift_apply(cv, S->s, &S->d_S->shift[0], st);
        launch_shift_apply(cv, z, &S->d_S->shift[1], st);
        S->launches += cl + 3;
    }
    QOCO_CUDA_TRY(cudaGetLastError());

    int status = QOCO_GPU_MAX_ITER;
    int it = 0;
    for (it = 0;; ++it) {
        {
            Phase ph(S, QOCO_GPU_PHASE_ROW, st);
            if (B) {
                IPMScalars tol;
                tol.abstol = S->st.abstol; tol.reltol = S->st.reltol;
                tol.abstol_inacc = S->st.abstol_inacc; tol.reltol_inacc = S->st.reltol_inacc;
                S->launches += launch_batch_residual(S->kv, S->bv, S->batch_L, S->xyz, S->s, S->d_c, S->d_b,
                                                     S->d_h, S->r, S->b_aux, it, tol, S->d_S, st);
            } else {
                const int nl = launch_residual(S->kv, S->lpr, S->xyz, S->s, S->d_c, S->d_b, S->d_h, S->r,
                                               S->partial, S->partial_cap, S->d_S, st);
                if (nl < 0) return QOCO_GPU_ERR_INVALID_ARG;
                S->launches += nl;
            }
        }
        QOCO_CUDA_TRY(cudaGetLastError());
        if ((rc = sync_scalars(S, st))) return rc;
        const IPMScalars& h = *S->h_S;
        S->info.pobj = h.pobj;
        S->info.dobj = h.dobj;
        S->info.gap = h.gap;
        S->info.pres = std::max(h.ry_inf, h.rz_inf);
        S->info.dres = h.rx_inf;
        S->info.iters = it;
        if (S->st.verbose)
            printf("%3d  pobj %+.8e  dobj %+.8e  gap %.2e  pres %.2e  dres %.2e  alpha %.3f\n", it, h.pobj,
                   h.dobj, h.gap, S->info.pres, h.rx_inf, it ? h.alpha : 0.0);
        if (h.nonfinite) { status = QOCO_GPU_ERR_NUMERICAL; break; }
        if (h.converged) { status = QOCO_GPU_SOLVED; break; }
        if (it >= S->st.max_iter) {
            status = h.converged_inacc ? QOCO_GPU_SOLVED_INACCURATE : QOCO_GPU_MAX_ITER;
            break;
        }
        // NT scaling, −W² into the KKT values, factor
        {
            Phase ph(S, QOCO_GPU_PHASE_CONE, st);
            S->launches += launch_nt_scaling(cv, S->s, z, S->wbar, S->eta, S->lam, S->d_val, S->d_w2slot,
                                             S->d_w2ptr, st);
        }
        // FP32 large fronts again after an FP64 escalation, unless the last two failed
        S->plan.big_fp32 = S->mixed_ok && S->fp32_fail_streak < 2;
        // predictor right-hand side first: the factorisation can run its forward sweep
        if (n + p) { k_neg_copy<<<grid(n + p), 256, 0, st>>>(S->rhs, S->r, n + p); S->launches++; }
        if (m) {
            Phase ph(S, QOCO_GPU_PHASE_CONE, st);
            launch_rhs_z(cv, S->lam, S->wbar, S->eta, S->r + n + p, nullptr, nullptr, nullptr, false, S->t,
                         S->t1, S->t2, S->rhs + n + p, st);
            S->launches += cl;
        }
        if ((rc = factor_now(S, st, S->rhs))) return rc;
        // predictor
        if ((rc = solve_refine(S, S->rhs, S->d_aff, st))) return rc;
        if (m) {
            Phase ph(S, QOCO_GPU_PHASE_CONE, st);
            launch_ds(cv, S->wbar, S->eta, S->t, S->d_aff + n + p, S->t1, S->ds_aff, st);
            if (B) {
                S->launches += cl + launch_batch_max_step(cv, S->bv, S->s, S->ds_aff, z, S->d_aff + n + p,
                                                          S->b_items, st);
            } else {
                launch_max_step(cv, S->s, S->ds_aff, z, S->d_aff + n + p, INFINITY, S->partial,
                                &S->d_S->alpha_max, st);
                S->launches += cl + 2;
            }
        } else {
            k_set<<<1, 1, 0, st>>>(&S->d_S->alpha_max, INFINITY);  // no cone limits the step
            S->launches++;
        }
        if (B) S->launches += launch_batch_sigma(S->bv, st);
        else { k_sigma<<<1, 1, 0, st>>>(S->d_S, 3.0); S->launches++; }
        // corrector
        if (m) {
            Phase ph(S, QOCO_GPU_PHASE_CONE, st);
            launch_rhs_z(cv, S->lam, S->wbar, S->eta, S->r + n + p, S->ds_aff, S->d_aff + n + p,
                         B ? S->bv.sigma_mu : &S->d_S->sigma_mu, true, S->t, S->t1, S->t2, S->rhs + n + p, st);
            S->launches += cl;
        }
        if ((rc = solve_refine(S, S->rhs, S->d_cmb, st))) return rc;
        if (m) {
            Phase ph(S, QOCO_GPU_PHASE_CONE, st);
            launch_ds(cv, S->wbar, S->eta, S->t, S->d_cmb + n + p, S->t1, S->ds_cmb, st);
            if (B) {
                S->launches += cl + launch_batch_max_step(cv, S->bv, S->s, S->ds_cmb, z, S->d_cmb + n + p,
                                                          S->b_items, st);
            } else {
                launch_max_step(cv, S->s, S->ds_cmb, z, S->d_cmb + n + p, INFINITY, S->partial,
                                &S->d_S->alpha_max, st);
                S->launches += cl + 2;
            }
        } else {
            k_set<<<1, 1, 0, st>>>(&S->d_S->alpha_max, INFINITY);
            S->launches++;
        }
        if (B) {
            S->launches += launch_batch_step(S->bv, S->st.step_fraction, S->xyz, S->s, S->d_cmb, S->ds_cmb, N,
                                             n + p, m, st);
        } else {
            k_alpha<<<1, 1, 0, st>>>(S->d_S);
            k_update<<<grid(std::max(N, m)), 256, 0, st>>>(S->xyz, S->s, S->d_cmb, S->ds_cmb, S->d_S, N, m);
            S->launches += 2;
        }
        QOCO_CUDA_TRY(cudaGetLastError());
    }
    return status;
}

void fill_info(const qoco_gpu_solver* S, qoco_gpu_info* info) {
    *info = S->info;
    info->kkt_dim = S->N;
    info->kkt_nnz = S->K.nnz();
    info->l_nnz = S->S.l_nnz;
    info->front_entries = S->S.front_entries;
    info->factor_flops = S->S.flops;
    info->n_supernodes = S->S.ns;
    info->n_levels = S->S.n_levels;
    info->max_front = S->S.max_front;
    info->refine_steps = S->refine_steps;
    info->last_backward_error = S->last_berr;
    info->kernel_launches = S->launches;
    info->h2d_bytes = S->h2d_bytes;
    info->d2h_bytes = S->d2h_bytes;
    info->fp32_factors = S->fp32_factors;
    info->fp64_escalations = S->fp64_escalations;
    info->fp32_floor_raises = S->fp32_floor_raises;
    info->krylov_steps = S->krylov_steps;
    info->batch_warps = S->fused_nw;
    info->batch_thread_fronts = S->fused_nw ? S->fused_split : 0;
    info->batch_warps_per_sm = S->fused_nw ? (S->fused_dense ? 32 : 16) : 0;
    snprintf(info->message, sizeof info->message, "%s", S->msg.c_str());
}

int analyze_common(int n, int m, int p, const qoco_csc* P, const double* c, const qoco_csc* A,
                   const double* b, const qoco_csc* G, const double* h, int l, int nsoc, const int* q,
                   const qoco_gpu_settings* settings, bool check_vectors, qoco_gpu_settings* st,
                   KKTPattern* K, Symbolic* Y, std::string* msg, double* t_analysis, int* used,
                   int trees = 1) {
    if (settings) *st = *settings;
    else qoco_gpu_default_settings(st);
    int rc = validate_problem(n, m, p, P, c, A, b, G, h, l, nsoc, q, check_vectors, msg);
    if (rc) return rc;
    const double t0 = now_s();
    build_kkt_pattern(K, n, m, p, P, A, G, l, nsoc, q);
    *used = analyze(*K, *st, Y, trees);
    *t_analysis = now_s() - t0;
    return 0;
}

// ---- batches --------------------------------------------------------------------
// an analysis made before the solver exists (a batch's, from its instance patterns)
struct Prebuilt {
    KKTPattern K;
    Symbolic Y;
    int used = 0;
    double t_analysis = 0.0;
};

struct Stacked {
    int n = 0, m = 0, p = 0, l = 0, nsoc = 0;
    std::vector<int> Pp{0}, Pi, Ap{0}, Ai, Gp{0}, Gi, q;
    std::vector<double> Pv, Av, Gv, c, b, h;
    std::vector<int> xo{0}, yo{0}, lo{0}, ko{0}, so{0};
    std::vector<double> nu, c_inf, b_inf, h_inf;
};

bool csc_present(const qoco_csc* M) { return M && M->colptr && M->n_cols > 0; }

// Block-diagonal stack of the instances: x and y in instance order; the cone's rows are
// every instance's orthant rows (instance order), then every instance's SOC rows.
// Without vectors (c == nullptr: an analysis only) c, b and h are left zero.
int stack_batch(int nb, const int* n, const int* m, const int* p, const qoco_csc* P, const double* const* c,
                const qoco_csc* A, const double* const* b, const qoco_csc* G, const double* const* h,
                const int* l, const int* nsoc, const int* const* q, Stacked* T, std::string* msg) {
    const bool vec = c != nullptr;
    for (int i = 0; i < nb; ++i) {
        if (m[i] <= 0) {
            // the per-instance barrier parameter μ = sᵀz / ν needs ν = l + nsoc > 0
            *msg = "instance " + std::to_string(i) + ": a batch instance needs cone rows (m > 0)";
            return QOCO_GPU_ERR_NOT_IMPLEMENTED;
        }
        int rc = validate_problem(n[i], m[i], p[i], csc_present(&P[i]) ? &P[i] : nullptr, vec ? c[i] : nullptr,
                                  p[i] ? &A[i] : nullptr, vec ? b[i] : nullptr, &G[i], vec ? h[i] : nullptr, l[i],
                                  nsoc[i], q[i], vec, msg);
        if (rc) {
            *msg = "instance " + std::to_string(i) + ": " + *msg;
            return rc;
        }
        T->n += n[i]; T->p += p[i]; T->m += m[i]; T->l += l[i]; T->nsoc += nsoc[i];
    }
    const int L = T->l;
    for (int i = 0; i < nb; ++i) {
        T->xo.push_back(T->xo.back() + n[i]);
        T->yo.push_back(T->yo.back() + p[i]);
        T->lo.push_back(T->lo.back() + l[i]);
        T->ko.push_back(T->ko.back() + nsoc[i]);
        T->so.push_back(T->so.back() + m[i] - l[i]);
    }
    T->h.assign(T->m, 0.0);
    for (int i = 0; i < nb; ++i) {
        const int xo = T->xo[i], yo = T->yo[i], lo = T->lo[i], so = T->so[i];
        double ci = 0.0, bi = 0.0, hi = 0.0;
        for (int j = 0; j < n[i]; ++j) {
            const double cj = vec ? c[i][j] : 0.0;
            T->c.push_back(cj);
            ci = std::max(ci, std::fabs(cj));
            // column j of the instance's P, A and G
            if (csc_present(&P[i]))
                for (int t = P[i].colptr[j]; t < P[i].colptr[j + 1]; ++t) {
                    T->Pi.push_back(xo + P[i].rowidx[t]);
                    T->Pv.push_back(P[i].val[t]);
                }
            T->Pp.push_back((int)T->Pi.size());
            if (p[i])
                for (int t = A[i].colptr[j]; t < A[i].colptr[j + 1]; ++t) {
                    T->Ai.push_back(yo + A[i].rowidx[t]);
                    T->Av.push_back(A[i].val[t]);
                }
            T->Ap.push_back((int)T->Ai.size());
            for (int t = G[i].colptr[j]; t < G[i].colptr[j + 1]; ++t) {
                const int r = G[i].rowidx[t];
                T->Gi.push_back(r < l[i] ? lo + r : L + so + (r - l[i]));
                T->Gv.push_back(G[i].val[t]);
            }
            T->Gp.push_back((int)T->Gi.size());
        }
        for (int j = 0; j < p[i]; ++j) {
            const double bj = vec ? b[i][j] : 0.0;
            T->b.push_back(bj);
            bi = std::max(bi, std::fabs(bj));
        }
        for (int r = 0; r < m[i]; ++r) {
            const double hr = vec ? h[i][r] : 0.0;
            T->h[r < l[i] ? lo + r : L + so + (r - l[i])] = hr;
            hi = std::max(hi, std::fabs(hr));
        }
        for (int k = 0; k < nsoc[i]; ++k) T->q.push_back(q[i][k]);
        T->nu.push_back((double)(l[i] + nsoc[i]));
        T->c_inf.push_back(ci);
        T->b_inf.push_back(bi);
        T->h_inf.push_back(hi);
    }
    return 0;
}

// The KKT pattern and symbolic analysis of a batch's stack from one analysis per distinct
// instance pattern (equal sizes, cone dimensions and P, A, G sparsity patterns): instances
// of the same model (an MPC horizon, say) are ordered and analysed once, and the stack's
// arrays are their relabelled copies (stack_analysis), the same as analysing the stack
// with the instances' orderings concatenated.  Returns the ordering used.
int batch_analysis(int nb, const int* n, const int* m, const int* p, const qoco_csc* P, const qoco_csc* A,
                   const qoco_csc* G, const int* l, const int* nsoc, const int* const* q, const Stacked& T,
                   const qoco_gpu_settings& st, KKTPattern* K, Symbolic* Y) {
    auto pmat = [&](int i) -> const qoco_csc* { return csc_present(&P[i]) && P[i].nnz > 0 ? &P[i] : nullptr; };
    auto amat = [&](int i) -> const qoco_csc* { return p[i] ? &A[i] : nullptr; };
    auto gmat = [&](int i) -> const qoco_csc* { return m[i] ? &G[i] : nullptr; };
    auto same_pattern = [&](const qoco_csc* a, const qoco_csc* b, int ncol) {
        if (!a || !b) return a == b;
        return a->nnz == b->nnz && std::equal(a->colptr, a->colptr + ncol + 1, b->colptr) &&
               std::equal(a->rowidx, a->rowidx + a->nnz, b->rowidx);
    };
    auto same = [&](int i, int r) {
        return n[i] == n[r] && m[i] == m[r] && p[i] == p[r] && l[i] == l[r] && nsoc[i] == nsoc[r] &&
               std::equal(q[i], q[i] + nsoc[i], q[r]) && same_pattern(pmat(i), pmat(r), n[i]) &&
               same_pattern(amat(i), amat(r), n[i]) && same_pattern(gmat(i), gmat(r), n[i]);
    };
    auto hash = [&](int i) {
        uint64_t h = 1469598103934665603ull;
        auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
        mix(n[i]); mix(m[i]); mix(p[i]); mix(l[i]); mix(nsoc[i]);
        for (int k = 0; k < nsoc[i]; ++k) mix(q[i][k]);
        for (const qoco_csc* M : {pmat(i), amat(i), gmat(i)}) {
            if (!M) { mix(~0ull); continue; }
            mix(M->nnz);
            for (int j = 0; j <= n[i]; ++j) mix(M->colptr[j]);
            for (int t = 0; t < M->nnz; ++t) mix(M->rowidx[t]);
        }
        return h;
    };
    std::vector<int> cls(nb), rep, count;
    std::map<uint64_t, std::vector<int>> by_hash;  // hash → pattern classes
    for (int i = 0; i < nb; ++i) {
        std::vector<int>& cand = by_hash[hash(i)];
        int c = -1;
        for (int k : cand)
            if (same(i, rep[k])) { c = k; break; }
        if (c < 0) {
            c = (int)rep.size();
            rep.push_back(i);
            count.push_back(0);
            cand.push_back(c);
        }
        cls[i] = c;
        ++count[c];
    }
    std::vector<KKTPattern> pats(rep.size());
    for (size_t c = 0; c < rep.size(); ++c) {
        const int r = rep[c];
        build_kkt_pattern(&pats[c], n[r], m[r], p[r], pmat(r), amat(r), gmat(r), l[r], nsoc[r], q[r]);
    }
    std::vector<std::vector<int>> perms;
    const int used = order_batch_patterns(pats, count, st, nb, &perms);
    std::vector<Symbolic> syms(rep.size());
    {
        // the patterns' own analyses, a few per host thread
        const int np = (int)rep.size();
        const int nth = std::max(1, std::min(np, (int)std::min(16u, std::max(1u, std::thread::hardware_concurrency()))));
        std::vector<std::thread> pool;
        auto work = [&](int t0) {
            for (int c = t0; c < np; c += nth) analyze(pats[c], st, &syms[c], 1, &perms[c], used);
        };
        for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
        work(0);
        for (auto& t : pool) t.join();
    }
    StackLayout L;
    L.n = T.n; L.p = T.p; L.m = T.m; L.l = T.l;
    L.xo = T.xo; L.yo = T.yo; L.lo = T.lo; L.so = T.so; L.ko = T.ko;
    L.Poff.resize(nb + 1);
    L.Aoff.resize(nb + 1);
    L.Goff.resize(nb + 1);
    for (int i = 0; i <= nb; ++i) {
        // an instance's data starts at the stack column of its first x
        L.Poff[i] = T.Pp[T.xo[i]];
        L.Aoff[i] = T.Ap[T.xo[i]];
        L.Goff[i] = T.Gp[T.xo[i]];
    }
    stack_analysis(pats, syms, cls, L, T.q, T.Pv.data(), T.Av.data(), T.Gv.data(), K, Y);
    return used;
}

// Per-instance schedules of a batch's factorisation and solves (see launch_inst_factor):
// when every front fits one warp, each instance's supernodes are listed level by level,
// thread fronts (order ≤ kThreadFront, schedule 0 only) before warp fronts, and the
// instances are queued by decreasing work Σ f²(c + 1).
int plan_batch_instances(qoco_gpu_solver* S, int nb, const std::vector<int>& row) {
    const Symbolic& Y = S->S;
    FactorPlan& P = S->plan;
    if (Y.ns == 0 || Y.max_front > kWarpFront || !P.groups.empty() || !P.big_s.empty()) return 0;
    std::vector<int> inst(Y.ns);
    int maxlev = 0;
    std::vector<double> work(nb, 0.0);
    for (int s = 0; s < Y.ns; ++s) {
        inst[s] = row[Y.perm[Y.sn_first[s]]];
        for (int j = Y.sn_first[s]; j < Y.sn_first[s + 1]; ++j)
            if (row[Y.perm[j]] != inst[s]) return 0;  // a front spanning instances: keep the shared kernels
        maxlev = std::max(maxlev, Y.level[s]);
        const double f = Y.sn_nrow[s], c = Y.sn_ncol[s];
        work[inst[s]] += f * f * (c + 1.0);
    }
    // supernodes bucketed by (instance, level), postorder kept inside a bucket
    const int64_t nkey = (int64_t)nb * (maxlev + 1);
    std::vector<int64_t> cnt(nkey + 1, 0);
    for (int s = 0; s < Y.ns; ++s) cnt[(int64_t)inst[s] * (maxlev + 1) + Y.level[s] + 1]++;
    for (int64_t k = 0; k < nkey; ++k) cnt[k + 1] += cnt[k];
    std::vector<int> bucket(Y.ns);
    {
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (int s = 0; s < Y.ns; ++s) bucket[fill[(int64_t)inst[s] * (maxlev + 1) + Y.level[s]]++] = s;
    }
    P.ninst = nb;
    int rc;
    for (int v = 0; v < 2; ++v) {
        const int thr = v == 0 ? kThreadFront : 0;
        std::vector<int> lv_ptr(1, 0), ent, sched;
        sched.reserve(Y.ns);
        for (int i = 0; i < nb; ++i) {
            for (int L = 0; L <= maxlev; ++L) {
                const int64_t b0 = cnt[(int64_t)i * (maxlev + 1) + L], b1 = cnt[(int64_t)i * (maxlev + 1) + L + 1];
                if (b0 == b1) continue;
                const int t0 = (int)sched.size();
                for (int64_t e = b0; e < b1; ++e)
                    if (Y.sn_nrow[bucket[e]] <= thr) sched.push_back(bucket[e]);
                const int w0 = (int)sched.size();
                for (int64_t e = b0; e < b1; ++e)
                    if (Y.sn_nrow[bucket[e]] > thr) sched.push_back(bucket[e]);
                ent.push_back(t0);
                ent.push_back(w0);
                ent.push_back((int)sched.size());
            }
            lv_ptr.push_back((int)ent.size() / 3);
        }
        if ((rc = dcopy(S, &P.isched[v].d_lv_ptr, lv_ptr))) return rc;
        if ((rc = dcopy(S, &P.isched[v].d_ent, ent))) return rc;
        if ((rc = dcopy(S, &P.isched[v].d_sched, sched))) return rc;
    }
    std::vector<int> order(nb);
    for (int i = 0; i < nb; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    if ((rc = dcopy(S, &P.d_inst_order, order))) return rc;
    if ((rc = dalloc(S, &P.d_inst_next, 2))) return rc;
    if ((rc = plan_instances(P, Y.max_front))) return rc;
    P.inst_variant = S->st.batch_schedule;  // 0: chosen on the first factorisation
    return 0;
}

int batch_init(qoco_gpu_solver* S, int nb, const Stacked& T) {
    int rc;
    BatchView& B = S->bv;
    B.nb = nb;
    int* pi;
    double* pd;
    if ((rc = dcopy(S, &pi, T.xo))) return rc; B.xo = pi;
    if ((rc = dcopy(S, &pi, T.yo))) return rc; B.yo = pi;
    if ((rc = dcopy(S, &pi, T.lo))) return rc; B.lo = pi;
    if ((rc = dcopy(S, &pi, T.ko))) return rc; B.ko = pi;
    if ((rc = dcopy(S, &pi, T.so))) return rc; B.so = pi;
    if ((rc = dcopy(S, &pd, T.nu))) return rc; B.nu = pd;
    if ((rc = dcopy(S, &pd, T.c_inf))) return rc; B.c_inf = pd;
    if ((rc = dcopy(S, &pd, T.b_inf))) return rc; B.b_inf = pd;
    if ((rc = dcopy(S, &pd, T.h_inf))) return rc; B.h_inf = pd;
    // instance of every KKT row, of every orthant entry and of every SOC
    const int n = T.n, p = T.p, L = T.l;
    std::vector<int> row(n + p + T.m), orth(L), soc(T.nsoc);
    for (int i = 0; i < nb; ++i) {
        for (int j = T.xo[i]; j < T.xo[i + 1]; ++j) row[j] = i;
        for (int j = T.yo[i]; j < T.yo[i + 1]; ++j) row[n + j] = i;
        for (int j = T.lo[i]; j < T.lo[i + 1]; ++j) { row[n + p + j] = i; orth[j] = i; }
        for (int j = T.so[i]; j < T.so[i + 1]; ++j) row[n + p + L + j] = i;
        for (int k = T.ko[i]; k < T.ko[i + 1]; ++k) soc[k] = i;
    }
    if ((rc = dcopy(S, &pi, row))) return rc; B.inst_row = pi;
    const int bs = S->st.batch_schedule;
    const bool want_fused = bs == 0 || (bs >= 6 && bs <= 12);
    if ((bs >= 0 && bs < kSharedSchedule) || want_fused)
        if ((rc = plan_batch_instances(S, nb, row))) return rc;
    if (want_fused && S->plan.inst) {
        for (int nw : {1, 2, 4})
            for (int dense = 0; dense < 2; ++dense)
                if ((rc = batch_ipm_grid(nw, dense, S->st.mixed_precision != 0, S->plan.inst_fmax, nb,
                                         &S->fused_grid[fused_grid_index(nw, dense)])))
                    return rc;
        for (int g : S->fused_grid) S->fused = S->fused || g > 0;
        // schedules 7–12 fix the tile (warps per CTA 1, 1, 2, 2, 4, 4; 16 or 32 warps per
        // SM); a tile this batch cannot launch is left to the tuning
        if (bs >= 7) {
            const int nw = 1 << ((bs - 7) / 2), dense = (bs - 7) % 2;
            if (S->fused_grid[fused_grid_index(nw, dense)] > 0) {
                S->fused_nw = nw;
                S->fused_split = 1;
                S->fused_dense = dense;
            }
        }
    }
    // the factorisation entry points outside a batched solve (kkt_factor_at, backward)
    // use the shared kernels when the persistent kernel runs the solves
    if (want_fused) S->plan.inst_variant = kSharedSchedule;
    S->info.batch_schedule_used = S->fused ? 6 : S->plan.inst ? bs : kSharedSchedule;
    if (L) { if ((rc = dcopy(S, &pi, orth))) return rc; S->cv.inst_orth = pi; }
    if (T.nsoc) { if ((rc = dcopy(S, &pi, soc))) return rc; S->cv.inst_soc = pi; }
    double** vd[] = {&B.pobj, &B.dobj, &B.gap, &B.mu, &B.alpha_max, &B.sigma_mu, &B.alpha};
    for (double** v : vd) if ((rc = dalloc(S, v, nb))) return rc;
    if ((rc = dalloc(S, &B.res, 3 * (size_t)nb))) return rc;
    int** vi[] = {&B.conv, &B.conv_inacc, &B.nonfinite, &B.iters};
    for (int** v : vi) if ((rc = dalloc(S, v, nb))) return rc;
    if ((rc = dalloc(S, &S->b_items, 2 * (size_t)std::max(1, L + T.nsoc)))) return rc;
    if ((rc = dalloc(S, &S->b_shift, 2 * (size_t)nb))) return rc;
    if ((rc = dalloc(S, &S->b_aux, 3 * (size_t)(n + p + T.m)))) return rc;
    S->batch = true;
    S->batch_L = L;
    S->h_xo = T.xo; S->h_yo = T.yo; S->h_lo = T.lo; S->h_ko = T.ko; S->h_so = T.so;
    if (S->fused) {
        BatchIPMArgs& A = S->bargs;
        A.K = S->kv;
        A.C = S->cv;
        A.F = S->fv;
        A.B = B;
        A.L = L;
        A.order = S->plan.d_inst_order;
        A.next = S->plan.d_inst_next;
        A.w2slot = S->d_w2slot;
        A.w2ptr = S->d_w2ptr;
        A.kval = S->d_val;
        A.c = S->d_c; A.b = S->d_b; A.h = S->d_h;
        A.xyz = S->xyz; A.s = S->s;
        A.d_aff = S->d_aff; A.ds_aff = S->ds_aff; A.d_cmb = S->d_cmb; A.ds_cmb = S->ds_cmb;
        A.r = S->r; A.rhs = S->rhs; A.wbar = S->wbar; A.eta = S->eta; A.lam = S->lam;
        A.t = S->t; A.t1 = S->t1; A.t2 = S->t2;
        A.sol_w = S->sol_w; A.sol_xp = S->sol_xp; A.res = S->res;
        A.abstol = S->st.abstol; A.reltol = S->st.reltol;
        A.abstol_inacc = S->st.abstol_inacc; A.reltol_inacc = S->st.reltol_inacc;
        A.refine_tol = S->st.refine_tol; A.step_fraction = S->st.step_fraction;
        A.max_iter = S->st.max_iter; A.max_refine = S->st.max_refine;
        A.fmax = S->plan.inst_fmax;
        A.mixed = S->st.mixed_precision != 0;
    }
    return 0;
}

int setup_impl(qoco_gpu_solver** out, int n, int m, int p, const qoco_csc* P, const double* c,
               const qoco_csc* A, const double* b, const qoco_csc* G, const double* h, int l, int nsoc,
               const int* q, const qoco_gpu_settings* settings, int trees, Prebuilt* pre = nullptr);

}  // namespace

extern "C" {

void qoco_gpu_default_settings(qoco_gpu_settings* s) {
    if (!s) return;
    s->abstol = 1e-7;
    s->reltol = 1e-7;
    s->abstol_inacc = 1e-5;
    s->reltol_inacc = 1e-5;
    s->max_iter = 200;
    s->static_reg = 1e-8;
    s->dyn_reg_thresh = 1e-13;
    s->dyn_reg_value = 1e-7;
    s->max_refine = 10;
    s->refine_tol = 1e-10;
    s->step_fraction = 0.99;
    s->ordering = QOCO_GPU_ORDER_AUTO;
    s->nd_leaf = 0;
    s->wait_polls = 0;
    s->verbose = 0;
    s->mixed_precision = 0;
    s->mixed_reg = 0.0;
    s->batch_schedule = 0;
}

int qoco_gpu_analyze(int n, int m, int p, const qoco_csc* P, const qoco_csc* A, const qoco_csc* G, int l,
                     int nsoc, const int* q, const qoco_gpu_settings* settings, qoco_gpu_info* info,
                     int* perm, int* sn_ptr, int* sn_nrow, int* sn_level) {
    qoco_gpu_settings st;
    KKTPattern K;
    Symbolic Y;
    std::string msg;
    double ta = 0.0;
    int used = 0;
    int rc;
    try {
        rc = analyze_common(n, m, p, P, nullptr, A, nullptr, G, nullptr, l, nsoc, q, settings, false, &st,
                            &K, &Y, &msg, &ta, &used);
    } catch (const std::bad_alloc&) {
        return QOCO_GPU_ERR_OOM;
    }
    if (info) {
        memset(info, 0, sizeof *info);
        snprintf(info->message, sizeof info->message, "%s", msg.c_str());
    }
    if (rc) return rc;
    if (info) {
        info->analysis_time_s = ta;
        info->kkt_dim = K.N;
        info->kkt_nnz = K.nnz();
        info->l_nnz = Y.l_nnz;
        info->front_entries = Y.front_entries;
        info->factor_flops = Y.flops;
        info->n_supernodes = Y.ns;
        info->n_levels = Y.n_levels;
        info->max_front = Y.max_front;
        info->ordering_used = used;
    }
    if (perm) memcpy(perm, Y.perm.data(), sizeof(int) * K.N);
    if (sn_ptr) memcpy(sn_ptr, Y.sn_first.data(), sizeof(int) * (Y.ns + 1));
    if (sn_nrow) memcpy(sn_nrow, Y.sn_nrow.data(), sizeof(int) * Y.ns);
    if (sn_level) memcpy(sn_level, Y.level.data(), sizeof(int) * Y.ns);
    return 0;
}

int qoco_gpu_analyze_batch(int nb, const int* n, const int* m, const int* p, const qoco_csc* P,
                           const qoco_csc* A, const qoco_csc* G, const int* l, const int* nsoc,
                           const int* const* q, const qoco_gpu_settings* settings, qoco_gpu_info* info,
                           int* perm, int* sn_ptr, int* sn_nrow, int* sn_level) {
    if (nb <= 0 || !n || !m || !p || !P || !A || !G || !l || !nsoc || !q) return QOCO_GPU_ERR_INVALID_ARG;
    qoco_gpu_settings st;
    if (settings) st = *settings;
    else qoco_gpu_default_settings(&st);
    Stacked T;
    Prebuilt pre;
    std::string msg;
    int rc;
    const double t0 = now_s();
    try {
        rc = stack_batch(nb, n, m, p, P, nullptr, A, nullptr, G, nullptr, l, nsoc, q, &T, &msg);
        if (!rc && T.m == 0) rc = QOCO_GPU_ERR_NOT_IMPLEMENTED;
        if (!rc && st.ordering == QOCO_GPU_ORDER_NATURAL) {
            qoco_csc Pc{T.n, T.n, (int)T.Pi.size(), T.Pp.data(), T.Pi.data(), T.Pv.data()};
            qoco_csc Ac{T.p, T.n, (int)T.Ai.size(), T.Ap.data(), T.Ai.data(), T.Av.data()};
            qoco_csc Gc{T.m, T.n, (int)T.Gi.size(), T.Gp.data(), T.Gi.data(), T.Gv.data()};
            double ta = 0.0;
            rc = analyze_common(T.n, T.m, T.p, T.Pi.empty() ? nullptr : &Pc, nullptr, T.p ? &Ac : nullptr, nullptr,
                                &Gc, nullptr, T.l, T.nsoc, T.q.empty() ? nullptr : T.q.data(), &st, false, &st,
                                &pre.K, &pre.Y, &msg, &ta, &pre.used, nb);
        } else if (!rc) {
            pre.used = batch_analysis(nb, n, m, p, P, A, G, l, nsoc, q, T, st, &pre.K, &pre.Y);
        }
    } catch (const std::bad_alloc&) {
        rc = QOCO_GPU_ERR_OOM;
    }
    if (info) {
        memset(info, 0, sizeof *info);
        snprintf(info->message, sizeof info->message, "%s", msg.c_str());
    }
    if (rc) return rc;
    const KKTPattern& K = pre.K;
    const Symbolic& Y = pre.Y;
    if (info) {
        info->analysis_time_s = now_s() - t0;
        info->kkt_dim = K.N;
        info->kkt_nnz = K.nnz();
        info->l_nnz = Y.l_nnz;
        info->front_entries = Y.front_entries;
        info->factor_flops = Y.flops;
        info->n_supernodes = Y.ns;
        info->n_levels = Y.n_levels;
        info->max_front = Y.max_front;
        info->ordering_used = pre.used;
    }
    if (perm) memcpy(perm, Y.perm.data(), sizeof(int) * K.N);
    if (sn_ptr) memcpy(sn_ptr, Y.sn_first.data(), sizeof(int) * (Y.ns + 1));
    if (sn_nrow) memcpy(sn_nrow, Y.sn_nrow.data(), sizeof(int) * Y.ns);
    if (sn_level) memcpy(sn_level, Y.level.data(), sizeof(int) * Y.ns);
    return 0;
}

int qoco_gpu_setup(qoco_gpu_solver** out, int n, int m, int p, const qoco_csc* P, const double* c,
                   const qoco_csc* A, const double* b, const qoco_csc* G, const double* h, int l, int nsoc,
                   const int* q, const qoco_gpu_settings* settings) {
    return setup_impl(out, n, m, p, P, c, A, b, G, h, l, nsoc, q, settings, 1);
}

}  // extern "C"

namespace {

// qoco_gpu_setup for `trees` independent problems stacked block-diagonally (1: one problem)
int setup_impl(qoco_gpu_solver** out, int n, int m, int p, const qoco_csc* P, const double* c,
               const qoco_csc* A, const double* b, const qoco_csc* G, const double* h, int l, int nsoc,
               const int* q, const qoco_gpu_settings* settings, int trees, Prebuilt* pre) {
    if (!out) return QOCO_GPU_ERR_INVALID_ARG;
    *out = nullptr;
    const double t0 = now_s();
    qoco_gpu_solver* S = nullptr;
    try {
        S = new qoco_gpu_solver();
    } catch (const std::bad_alloc&) {
        return QOCO_GPU_ERR_OOM;
    }
    memset(&S->info, 0, sizeof S->info);
    double ta = 0.0;
    int used = 0;
    int rc;
    if (pre) {
        // a batch analysed from its instances' patterns (already validated)
        if (settings) S->st = *settings;
        else qoco_gpu_default_settings(&S->st);
        S->K = std::move(pre->K);
        S->S = std::move(pre->Y);
        ta = pre->t_analysis;
        used = pre->used;
        rc = 0;
    } else {
        try {
            rc = analyze_common(n, m, p, P, c, A, b, G, h, l, nsoc, q, settings, true, &S->st, &S->K, &S->S,
                                &S->msg, &ta, &used, trees);
        } catch (const std::bad_alloc&) {
            rc = QOCO_GPU_ERR_OOM;
        }
    }
    if (rc) {
        delete S;
        return rc;
    }
    S->n = n; S->m = m; S->p = p; S->N = n + p + m;
    rc = upload(S, c, b, h);
    if (rc) {
        qoco_gpu_cleanup(S);
        return rc;
    }
    S->info.analysis_time_s = ta;
    S->info.ordering_used = used;
    S->info.setup_time_s = now_s() - t0;
    *out = S;
    return 0;
}

}  // namespace

extern "C" {

int qoco_gpu_setup_batch(qoco_gpu_solver** out, int nb, const int* n, const int* m, const int* p,
                         const qoco_csc* P, const double* const* c, const qoco_csc* A, const double* const* b,
                         const qoco_csc* G, const double* const* h, const int* l, const int* nsoc,
                         const int* const* q, const qoco_gpu_settings* settings) {
    if (!out || nb <= 0 || !n || !m || !p || !P || !c || !A || !b || !G || !h || !l || !nsoc || !q)
        return QOCO_GPU_ERR_INVALID_ARG;
    *out = nullptr;
    const double t0 = now_s();
    Stacked T;
    std::string msg;
    int rc;
    try {
        rc = stack_batch(nb, n, m, p, P, c, A, b, G, h, l, nsoc, q, &T, &msg);
    } catch (const std::bad_alloc&) {
        rc = QOCO_GPU_ERR_OOM;
    }
    if (rc) return rc;
    const double t_stacked = now_s();
    if (T.m == 0) return QOCO_GPU_ERR_NOT_IMPLEMENTED;  // a batch needs cone rows
    qoco_csc Pc{T.n, T.n, (int)T.Pi.size(), T.Pp.data(), T.Pi.data(), T.Pv.data()};
    qoco_csc Ac{T.p, T.n, (int)T.Ai.size(), T.Ap.data(), T.Ai.data(), T.Av.data()};
    qoco_csc Gc{T.m, T.n, (int)T.Gi.size(), T.Gp.data(), T.Gi.data(), T.Gv.data()};
    // one analysis per distinct instance pattern (the natural ordering is the stack's own)
    qoco_gpu_settings st;
    if (settings) st = *settings;
    else qoco_gpu_default_settings(&st);
    Prebuilt pre;
    const bool by_pattern = st.ordering != QOCO_GPU_ORDER_NATURAL;
    if (by_pattern) {
        const double ta = now_s();
        try {
            pre.used = batch_analysis(nb, n, m, p, P, A, G, l, nsoc, q, T, st, &pre.K, &pre.Y);
        } catch (const std::bad_alloc&) {
            return QOCO_GPU_ERR_OOM;
        }
        pre.t_analysis = now_s() - ta;
    }
    qoco_gpu_solver* S = nullptr;
    rc = setup_impl(&S, T.n, T.m, T.p, T.Pi.empty() ? nullptr : &Pc, T.c.data(), T.p ? &Ac : nullptr,
                    T.p ? T.b.data() : nullptr, &Gc, T.h.data(), T.l, T.nsoc, T.q.empty() ? nullptr : T.q.data(),
                    settings, nb, by_pattern ? &pre : nullptr);
    if (rc) return rc;
    const double t_device = S->info.setup_time_s;  // setup_impl: upload and launch plans
    const double t_init = now_s();
    try {
        rc = batch_init(S, nb, T);
    } catch (const std::bad_alloc&) {
        rc = QOCO_GPU_ERR_OOM;
    }
    if (rc) {
        qoco_gpu_cleanup(S);
        return rc;
    }
    S->info.setup_time_s = now_s() - t0;
    if (S->st.verbose >= 2)
        printf("batch set-up %.3f s: stack %.3f, analysis %.3f, upload and plans %.3f, batch plans %.3f\n",
               S->info.setup_time_s, t_stacked - t0, S->info.analysis_time_s,
               t_device - (by_pattern ? 0.0 : S->info.analysis_time_s),
               now_s() - t_init);
    *out = S;
    return 0;
}

int qoco_gpu_batch_size(const qoco_gpu_solver* S) { return S && S->batch ? S->bv.nb : 0; }

int qoco_gpu_batch_offsets(const qoco_gpu_solver* S, int* xo, int* yo, int* lo, int* ko, int* so) {
    if (!S || !S->batch) return QOCO_GPU_ERR_INVALID_ARG;
    const size_t k = S->h_xo.size();
    if (xo) memcpy(xo, S->h_xo.data(), sizeof(int) * k);
    if (yo) memcpy(yo, S->h_yo.data(), sizeof(int) * k);
    if (lo) memcpy(lo, S->h_lo.data(), sizeof(int) * k);
    if (ko) memcpy(ko, S->h_ko.data(), sizeof(int) * k);
    if (so) memcpy(so, S->h_so.data(), sizeof(int) * k);
    return 0;
}

int qoco_gpu_batch_info(const qoco_gpu_solver* S, int* status, int* iters, double* pobj, double* dobj,
                        double* gap) {
    if (!S || !S->batch) return QOCO_GPU_ERR_INVALID_ARG;
    const int nb = S->bv.nb;
    std::vector<int> cv(nb), ci(nb), nf(nb), it(nb);
    QOCO_CUDA_TRY(cudaDeviceSynchronize());
    QOCO_CUDA_TRY(cudaMemcpy(cv.data(), S->bv.conv, sizeof(int) * nb, cudaMemcpyDeviceToHost));
    QOCO_CUDA_TRY(cudaMemcpy(ci.data(), S->bv.conv_inacc, sizeof(int) * nb, cudaMemcpyDeviceToHost));
    QOCO_CUDA_TRY(cudaMemcpy(nf.data(), S->bv.nonfinite, sizeof(int) * nb, cudaMemcpyDeviceToHost));
    QOCO_CUDA_TRY(cudaMemcpy(it.data(), S->bv.iters, sizeof(int) * nb, cudaMemcpyDeviceToHost));
    if (status)
        for (int i = 0; i < nb; ++i)
            status[i] = cv[i] ? QOCO_GPU_SOLVED
                              : nf[i] ? QOCO_GPU_ERR_NUMERICAL
                                      : ci[i] ? QOCO_GPU_SOLVED_INACCURATE : QOCO_GPU_MAX_ITER;
    if (iters)
        for (int i = 0; i < nb; ++i) iters[i] = cv[i] ? it[i] : S->info.iters;
    if (pobj) QOCO_CUDA_TRY(cudaMemcpy(pobj, S->bv.pobj, sizeof(double) * nb, cudaMemcpyDeviceToHost));
    if (dobj) QOCO_CUDA_TRY(cudaMemcpy(dobj, S->bv.dobj, sizeof(double) * nb, cudaMemcpyDeviceToHost));
    if (gap) QOCO_CUDA_TRY(cudaMemcpy(gap, S->bv.gap, sizeof(double) * nb, cudaMemcpyDeviceToHost));
    return 0;
}

int qoco_gpu_solve(qoco_gpu_solver* S, void* stream) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const double t0 = now_s();
    S->launches = 0;
    S->d2h_bytes = 0;
    int status = run_solve(S, st);
    if (status == QOCO_GPU_ERR_CUDA || status == QOCO_GPU_ERR_OOM) S->msg = g_cuda_msg;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && status >= 0) status = cuda_fail(e, "stream sync", __FILE__, __LINE__);
    S->info.status = status;
    S->info.solve_time_s = now_s() - t0;
    S->have_solution = status >= 0;
    return status;
}

int qoco_gpu_get_solution(const qoco_gpu_solver* S, double* x, double* s, double* y, double* z,
                          qoco_gpu_info* info) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    QOCO_CUDA_TRY(cudaDeviceSynchronize());
    if (x) QOCO_CUDA_TRY(cudaMemcpy(x, S->xyz, sizeof(double) * S->n, cudaMemcpyDeviceToHost));
    if (y && S->p) QOCO_CUDA_TRY(cudaMemcpy(y, S->xyz + S->n, sizeof(double) * S->p, cudaMemcpyDeviceToHost));
    if (z && S->m)
        QOCO_CUDA_TRY(cudaMemcpy(z, S->xyz + S->n + S->p, sizeof(double) * S->m, cudaMemcpyDeviceToHost));
    if (s && S->m) QOCO_CUDA_TRY(cudaMemcpy(s, S->s, sizeof(double) * S->m, cudaMemcpyDeviceToHost));
    if (info) fill_info(S, info);
    return 0;
}

int qoco_gpu_solution_device(const qoco_gpu_solver* S, const double** x, const double** s, const double** y,
                             const double** z) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    if (x) *x = S->xyz;
    if (y) *y = S->xyz + S->n;
    if (z) *z = S->xyz + S->n + S->p;
    if (s) *s = S->s;
    return 0;
}

int qoco_gpu_copy_solution(const qoco_gpu_solver* S, double* x, double* s, double* y, double* z, void* stream) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (x && S->n) QOCO_CUDA_TRY(cudaMemcpyAsync(x, S->xyz, sizeof(double) * S->n, k, st));
    if (y && S->p) QOCO_CUDA_TRY(cudaMemcpyAsync(y, S->xyz + S->n, sizeof(double) * S->p, k, st));
    if (z && S->m) QOCO_CUDA_TRY(cudaMemcpyAsync(z, S->xyz + S->n + S->p, sizeof(double) * S->m, k, st));
    if (s && S->m) QOCO_CUDA_TRY(cudaMemcpyAsync(s, S->s, sizeof(double) * S->m, k, st));
    return 0;
}

int qoco_gpu_get_info(const qoco_gpu_solver* S, qoco_gpu_info* info) {
    if (!S || !info) return QOCO_GPU_ERR_INVALID_ARG;
    fill_info(S, info);
    return 0;
}

namespace {

// v ← K̂⁻ᵀ g by refinement preconditioned with the current factor (see the header);
// returns true when the backward error reached the refinement target
int adjoint_refine(qoco_gpu_solver* S, const double* g, double* v, bool* ok, cudaStream_t st) {
    const int n = S->n, p = S->p, m = S->m, N = S->N;
    double* rp = S->d_cmb;
    double* z = S->xyz + n + p;
    const int64_t nw2 = (int64_t)S->K.w2_slot.size();
    if (nw2) k_w2_zero<<<(unsigned)((nw2 + 255) / 256), 256, 0, st>>>(S->d_val, S->d_w2slot, nw2);
    ++S->launches;
    int rc = tri_solve(S, g, v, false, st);
    if (rc) return rc;
    const int max_steps = std::max(3 * S->st.max_refine, 10);
    double best = INFINITY;
    int stall = 0;
    *ok = false;
    for (int steps = 0;; ++steps) {
        if (m) {
            launch_div(S->cv, z, v + n + p, S->t1, st);
            launch_prod(S->cv, S->s, S->t1, S->t2, st);
            S->launches += 2 * cone_launch_count(S->cv);
        }
        k_adj_rhs<<<grid(N), 256, 0, st>>>(rp, g, m ? S->t2 : nullptr, n + p, N);
        ++S->launches;
        const int nl = launch_spmv_res(S->kv, S->lpr, v, rp, S->res, S->partial, S->partial_cap, S->d_S, st);
        if (nl < 0) return QOCO_GPU_ERR_INVALID_ARG;
        S->launches += nl;
        QOCO_CUDA_TRY(cudaGetLastError());
        if ((rc = sync_scalars(S, st))) return rc;
        if (S->h_S->bar_err) return QOCO_GPU_ERR_DEVICE_TIMEOUT;
        const double berr = S->h_S->berr;
        S->adj_steps = steps;
        S->adj_berr = berr;
        if (!std::isfinite(berr)) return 0;
        if (berr <= S->st.refine_tol) { *ok = true; return 0; }
        if (berr < 0.5 * best) { best = berr; stall = 0; }
        else if (++stall >= 4) return 0;
        if (steps >= max_steps) return 0;
        if ((rc = tri_solve(S, S->res, v, true, st))) return rc;
    }
}

}  // namespace

int qoco_gpu_backward(qoco_gpu_solver* S, const double* dx, const double* dy, const double* dz, double* dP_val,
                      double* dc, double* dA_val, double* db, double* dG_val, double* dh, void* stream) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    if (!S->have_solution || !S->have_factor) return QOCO_GPU_ERR_NO_FACTOR;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = S->n, p = S->p, m = S->m, N = S->N;
    double* g = S->rhs;
    double* v = S->d_aff;
    QOCO_CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(double) * N, st));
    if (dx && n) QOCO_CUDA_TRY(cudaMemcpyAsync(g, dx, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    if (dy && p) QOCO_CUDA_TRY(cudaMemcpyAsync(g + n, dy, sizeof(double) * p, cudaMemcpyDeviceToDevice, st));
    if (dz && m) QOCO_CUDA_TRY(cudaMemcpyAsync(g + n + p, dz, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
    int rc = reset_barrier(S, st);
    if (rc) return rc;
    S->adj_refactored = 0;
    bool ok = false;
    if ((rc = adjoint_refine(S, g, v, &ok, st))) return rc;
    if (!ok && m) {
        // refactor once at the final iterate's NT scaling, then refine again
        S->launches += launch_nt_scaling(S->cv, S->s, S->xyz + n + p, S->wbar, S->eta, S->lam, S->d_val,
                                         S->d_w2slot, S->d_w2ptr, st);
        if ((rc = factor_now(S, st))) return rc;
        S->adj_refactored = 1;
        if ((rc = adjoint_refine(S, g, v, &ok, st))) return rc;
    }
    if (!ok) return QOCO_GPU_ERR_NUMERICAL;
    const int64_t nd = S->K.nnzP + S->K.nnzA + S->K.nnzG;
    if (nd && (dP_val || dA_val || dG_val)) {
        k_adj_data_grad<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(S->d_adj_a, S->d_adj_b, nd, S->K.nnzP,
                                                                      S->K.nnzA, S->xyz, v, dP_val, dA_val, dG_val);
        ++S->launches;
    }
    k_adj_vec_grad<<<grid(N), 256, 0, st>>>(v, dc, db, dh, n, p, m);
    ++S->launches;
    QOCO_CUDA_TRY(cudaGetLastError());
    QOCO_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int qoco_gpu_backward_info(const qoco_gpu_solver* S, int* refine_steps, double* backward_error, int* refactored) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    if (refine_steps) *refine_steps = S->adj_steps;
    if (backward_error) *backward_error = S->adj_berr;
    if (refactored) *refactored = S->adj_refactored;
    return 0;
}

int qoco_gpu_update_data(qoco_gpu_solver* S, const double* P_val, const double* c, const double* A_val,
                         const double* b, const double* G_val, const double* h, int on_device, void* stream) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const KKTPattern& K = S->K;
    const int n = S->n, p = S->p, m = S->m;
    if (!on_device) {
        auto finite = [](const double* v, int64_t len) {
            for (int64_t i = 0; v && i < len; ++i)
                if (!std::isfinite(v[i])) return false;
            return true;
        };
        if (!finite(P_val, K.nnzP) || !finite(c, n) || !finite(A_val, K.nnzA) || !finite(b, p) ||
            !finite(G_val, K.nnzG) || !finite(h, m)) {
            S->msg = "update_data: non-finite value";
            return QOCO_GPU_ERR_NONFINITE_DATA;
        }
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // matrix values: host values are staged through the work vectors' storage so that one
    // scatter kernel serves both cases
    const double* src[3] = {P_val, A_val, G_val};
    const int64_t len[3] = {K.nnzP, K.nnzA, K.nnzG};
    double* dev[3] = {nullptr, nullptr, nullptr};
    std::vector<void*> tmp;
    for (int k = 0; k < 3; ++k) {
        if (!src[k] || !len[k]) continue;
        if (on_device) { dev[k] = const_cast<double*>(src[k]); continue; }
        void* d = nullptr;
        QOCO_CUDA_TRY(cudaMallocAsync(&d, sizeof(double) * len[k], st));
        tmp.push_back(d);
        QOCO_CUDA_TRY(cudaMemcpyAsync(d, src[k], sizeof(double) * len[k], kind, st));
        S->h2d_bytes += (int64_t)sizeof(double) * len[k];
        dev[k] = (double*)d;
    }
    if (S->n_data_slot && (dev[0] || dev[1] || dev[2])) {
        k_scatter_data<<<(unsigned)((S->n_data_slot + 255) / 256), 256, 0, st>>>(
            S->d_val, S->d_data_slot, S->d_data_src, S->n_data_slot, dev[0], dev[1], dev[2], K.nnzP, K.nnzA);
    }
    if (c && n) QOCO_CUDA_TRY(cudaMemcpyAsync(S->d_c, c, sizeof(double) * n, kind, st));
    if (b && p) QOCO_CUDA_TRY(cudaMemcpyAsync(S->d_b, b, sizeof(double) * p, kind, st));
    if (h && m) QOCO_CUDA_TRY(cudaMemcpyAsync(S->d_h, h, sizeof(double) * m, kind, st));
    if (!on_device) S->h2d_bytes += (int64_t)sizeof(double) * ((c ? n : 0) + (b ? p : 0) + (h ? m : 0));
    k_data_norms<<<1, 256, 0, st>>>(S->d_c, S->d_b, S->d_h, n, p, m, S->d_S);
    for (void* d : tmp) QOCO_CUDA_TRY(cudaFreeAsync(d, st));
    QOCO_CUDA_TRY(cudaGetLastError());
    S->have_solution = false;
    S->have_factor = false;
    return 0;
}

int qoco_gpu_set_profiling(qoco_gpu_solver* S, int on) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    QOCO_CUDA_TRY(cudaDeviceSynchronize());
    S->prof.flush();
    if (on < 0 || on > 2) return QOCO_GPU_ERR_INVALID_ARG;
    S->prof.on = on != 0;
    S->prof.factor_only = on == 2;
    memset(&S->prof.tot, 0, sizeof S->prof.tot);
    return 0;
}

int qoco_gpu_get_profile(const qoco_gpu_solver* S, qoco_gpu_profile* out) {
    if (!S || !out) return QOCO_GPU_ERR_INVALID_ARG;
    *out = S->prof.tot;
    return 0;
}

int qoco_gpu_cleanup(qoco_gpu_solver* S) {
    if (!S) return 0;
    for (auto& g : S->fgraph) if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& g : S->sgraphs) if (g.exec) cudaGraphExecDestroy(g.exec);
    if (S->bgraph.exec) cudaGraphExecDestroy(S->bgraph.exec);
    if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
    for (void* p : S->allocs) cudaFree(p);
    if (S->h_S) cudaFreeHost(S->h_S);
    delete S;
    return 0;
}

int qoco_gpu_kkt_factor_at(qoco_gpu_solver* S, const double* s, const double* z, void* stream) {
    if (!S || (S->m && (!s || !z))) return QOCO_GPU_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    S->launches += launch_nt_scaling(S->cv, s, z, S->wbar, S->eta, S->lam, S->d_val, S->d_w2slot, S->d_w2ptr, st);
    S->plan.big_fp32 = S->st.mixed_precision != 0 && S->plan.max_big_f > 0 && S->plan.big_work32;
    int rc = factor_now(S, st);
    if (rc) return rc;
    QOCO_CUDA_TRY(cudaStreamSynchronize(st));
    return 0;
}

int qoco_gpu_kkt_solve(qoco_gpu_solver* S, const double* r, double* x, int* refine_steps,
                       double* backward_error, void* stream) {
    if (!S || !r || !x) return QOCO_GPU_ERR_INVALID_ARG;
    if (!S->have_factor) return QOCO_GPU_ERR_NO_FACTOR;
    cudaStream_t st = (cudaStream_t)stream;
    const int before = S->refine_steps;
    int rc = reset_barrier(S, st);
    if (rc) return rc;
    rc = solve_refine(S, r, x, st);
    if (rc) return rc;
    QOCO_CUDA_TRY(cudaStreamSynchronize(st));
    if (refine_steps) *refine_steps = S->refine_steps - before;
    if (backward_error) *backward_error = S->last_berr;
    return 0;
}

int qoco_gpu_get_kkt(const qoco_gpu_solver* S, int64_t* rowptr, int* colidx, double* val) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    QOCO_CUDA_TRY(cudaDeviceSynchronize());
    if (rowptr) memcpy(rowptr, S->K.rowptr.data(), sizeof(int64_t) * (S->N + 1));
    if (colidx) memcpy(colidx, S->K.colidx.data(), sizeof(int) * S->K.nnz());
    if (val) QOCO_CUDA_TRY(cudaMemcpy(val, S->d_val, sizeof(double) * S->K.nnz(), cudaMemcpyDeviceToHost));
    return 0;
}

int qoco_gpu_get_factor_dense(const qoco_gpu_solver* S, int* perm, double* L, double* D) {
    if (!S) return QOCO_GPU_ERR_INVALID_ARG;
    const int N = S->N;
    if (N > 4096) return QOCO_GPU_ERR_INVALID_ARG;
    if (!S->have_factor) return QOCO_GPU_ERR_NO_FACTOR;
    const Symbolic& Y = S->S;
    std::vector<double> fr((size_t)Y.front_entries);
    QOCO_CUDA_TRY(cudaDeviceSynchronize());
    QOCO_CUDA_TRY(cudaMemcpy(fr.data(), S->fv.front, sizeof(double) * fr.size(), cudaMemcpyDeviceToHost));
    if (perm) memcpy(perm, Y.perm.data(), sizeof(int) * N);
    if (L) {
        memset(L, 0, sizeof(double) * (size_t)N * N);
        for (int i = 0; i < N; ++i) L[(size_t)i * N + i] = 1.0;
    }
    for (int s = 0; s < Y.ns; ++s) {
        const int f = Y.sn_nrow[s], c = Y.sn_ncol[s], first = Y.sn_first[s];
        const double* F = fr.data() + Y.front_off[s];
        const int* R = Y.rows.data() + Y.row_ptr[s];
        for (int k = 0; k < c; ++k) {
            if (D) D[first + k] = F[(size_t)k * f + k];
            if (L)
                for (int a = k + 1; a < f; ++a) L[(size_t)R[a] * N + first + k] = F[(size_t)k * f + a];
        }
    }
    return 0;
}

int qoco_gpu_cone_max_step_noalloc(const qoco_gpu_cones* C, const double* u, const double* du, double cap,
                                   double* alpha, void* stream) {
    if (!C || !alpha || (C->v.m && (!u || !du))) return QOCO_GPU_ERR_INVALID_ARG;
    return launch_max_step_noalloc(C->v, u, du, cap, alpha, (cudaStream_t)stream);
}

int qoco_gpu_selftest_wait_timeout(long long max_polls, void* stream) {
    if (max_polls < 1) return QOCO_GPU_ERR_INVALID_ARG;
    return selftest_wait_timeout(max_polls, (cudaStream_t)stream);
}

int qoco_gpu_get_pivot_reciprocals(const qoco_gpu_solver* S, double* dinv) {
    if (!S || !dinv) return QOCO_GPU_ERR_INVALID_ARG;
    if (!S->have_factor) return QOCO_GPU_ERR_NO_FACTOR;
    QOCO_CUDA_TRY(cudaDeviceSynchronize());
    QOCO_CUDA_TRY(cudaMemcpy(dinv, S->fv.dinv, sizeof(double) * S->N, cudaMemcpyDeviceToHost));
    return 0;
}

int qoco_gpu_cones_create(qoco_gpu_cones** out, int l, int nsoc, const int* q) {
    if (!out || l < 0 || nsoc < 0 || (nsoc && !q)) return QOCO_GPU_ERR_INVALID_ARG;
    *out = nullptr;
    auto* C = new (std::nothrow) qoco_gpu_cones();
    if (!C) return QOCO_GPU_ERR_OOM;
    std::vector<int> off(nsoc), dim(nsoc), sm, lg;
    int o = l;
    for (int k = 0; k < nsoc; ++k) {
        if (q[k] < 2) { delete C; return QOCO_GPU_ERR_INVALID_CONE; }
        off[k] = o;
        dim[k] = q[k];
        o += q[k];
        (q[k] <= kSmallCone ? sm : lg).push_back(k);
    }
    C->v.l = l; C->v.nsoc = nsoc; C->v.m = o;
    C->v.nsmall = (int)sm.size(); C->v.nlarge = (int)lg.size();
    std::vector<int>* src[4] = {&off, &dim, &sm, &lg};
    const int** dst[4] = {&C->v.off, &C->v.dim, &C->v.small, &C->v.large};
    for (int i = 0; i < 4; ++i) {
        int* d = nullptr;
        size_t bytes = std::max<size_t>(1, src[i]->size()) * sizeof(int);
        cudaError_t e = cudaMalloc((void**)&d, bytes);
        if (e == cudaSuccess && !src[i]->empty())
            e = cudaMemcpy(d, src[i]->data(), src[i]->size() * sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (d) cudaFree(d);
            qoco_gpu_cones_destroy(C);
            return cuda_fail(e, "cones_create", __FILE__, __LINE__);
        }
        C->allocs.push_back(d);
        *dst[i] = d;
    }
    *out = C;
    return 0;
}

int qoco_gpu_cones_destroy(qoco_gpu_cones* C) {
    if (!C) return 0;
    for (void* p : C->allocs) cudaFree(p);
    delete C;
    return 0;
}

int qoco_gpu_cone_nt_scaling(const qoco_gpu_cones* C, const double* s, const double* z, double* w, double* eta,
                             double* lambda, void* stream) {
    if (!C || (C->v.m && (!s || !z || !w || !lambda)) || (C->v.nsoc && !eta)) return QOCO_GPU_ERR_INVALID_ARG;
    launch_nt_scaling(C->v, s, z, w, eta, lambda, nullptr, nullptr, nullptr, (cudaStream_t)stream);
    QOCO_CUDA_TRY(cudaGetLastError());
    return 0;
}

int qoco_gpu_cone_product(const qoco_gpu_cones* C, const double* u, const double* v, double* out, void* stream) {
    if (!C || (C->v.m && (!u || !v || !out))) return QOCO_GPU_ERR_INVALID_ARG;
    launch_prod(C->v, u, v, out, (cudaStream_t)stream);
    QOCO_CUDA_TRY(cudaGetLastError());
    return 0;
}

int qoco_gpu_cone_division(const qoco_gpu_cones* C, const double* lam, const double* v, double* out,
                           void* stream) {
    if (!C || (C->v.m && (!lam || !v || !out))) return QOCO_GPU_ERR_INVALID_ARG;
    launch_div(C->v, lam, v, out, (cudaStream_t)stream);
    QOCO_CUDA_TRY(cudaGetLastError());
    return 0;
}

size_t qoco_gpu_cone_max_step_scratch_bytes(const qoco_gpu_cones* C) {
    if (!C) return 0;
    return sizeof(double) * (size_t)std::max(1, max_step_partials(C->v));
}

int qoco_gpu_cone_max_step(const qoco_gpu_cones* C, const double* u, const double* du, double cap,
                           double* alpha, void* scratch, void* stream) {
    if (!C || !alpha || !scratch || (C->v.m && (!u || !du))) return QOCO_GPU_ERR_INVALID_ARG;
    launch_max_step(C->v, u, du, nullptr, nullptr, cap, (double*)scratch, alpha, (cudaStream_t)stream);
    QOCO_CUDA_TRY(cudaGetLastError());
    return 0;
}

}  // extern "C"
