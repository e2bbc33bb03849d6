// Cone kernels of one interior-point iteration (K1–K4) and the stand-alone cone
// entry points of the C ABI.
#include "cone_kernels.h"

#include <algorithm>

#include <mutex>

#include "qoco_gpu.h"

namespace qoco {

// ---------------------------------------------------------------------------
// K1 + K2: NT scaling; −W² written into the KKT value array through the index map
// ---------------------------------------------------------------------------
__global__ void k_nt_scaling(ConeView c, ConeGrid g, const double* __restrict__ s,
                             const double* __restrict__ z, double* wbar, double* eta, double* lam,
                             double* kval, const int64_t* __restrict__ w2slot,
                             const int64_t* __restrict__ w2ptr) {
    ConeItem it;
    if (!cone_item(c, g, &it)) return;
    if (it.kind == 0) {
        const int i = it.idx;
        const double si = s[i], zi = z[i];
        wbar[i] = sqrt(si / zi);
        lam[i] = sqrt(si * zi);
        if (kval) kval[w2slot[i]] = -(si / zi);
        return;
    }
    const int k = it.idx, o = c.off[k], d = c.dim[k];
    double* kv = d > kWideCone ? nullptr : kval;  // wide cones: k_w2_wide writes the block
    const int64_t* slots = kv ? w2slot + c.l + w2ptr[k] : nullptr;
    if (it.kind == 1) soc_nt<1>(k, o, d, 0, s, z, wbar, eta, lam, kv, slots);
    else soc_nt<32>(k, o, d, it.lane, s, z, wbar, eta, lam, kv, slots);
}

// The −W² blocks of the wide SOCs, one thread per entry (coalesced slot reads):
// −η²(2 w̄_a w̄_b − J_ab), or −I for the initial point (identity != 0)
__global__ void k_w2_wide(ConeView c, const double* __restrict__ wbar, const double* __restrict__ eta,
                          double* __restrict__ kval, const int64_t* __restrict__ w2slot,
                          const int64_t* __restrict__ w2ptr, int identity) {
    for (int j = blockIdx.y; j < c.nwide; j += gridDim.y) {
        const int k = c.wide[j], d = c.dim[k], o = c.off[k];
        const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (e >= (int64_t)d * d) continue;
        const int a = (int)(e / d), b = (int)(e - (int64_t)a * d);
        const double J = (a == b) ? (a == 0 ? 1.0 : -1.0) : 0.0;
        double v;
        if (identity) {
            v = (a == b) ? -1.0 : 0.0;
        } else {
            const double e2 = eta[k] * eta[k];
            v = -e2 * (2.0 * wbar[o + a] * wbar[o + b] - J);
        }
        kval[w2slot[c.l + w2ptr[k] + e]] = v;
    }
}

// W = I in the KKT value array (initial point)
__global__ void k_w2_identity(ConeView c, ConeGrid g, double* kval, const int64_t* __restrict__ w2slot,
                              const int64_t* __restrict__ w2ptr) {
    ConeItem it;
    if (!cone_item(c, g, &it)) return;
    if (it.kind == 0) { kval[w2slot[it.idx]] = -1.0; return; }
    const int k = it.idx, d = c.dim[k];
    if (d > kWideCone) return;  // k_w2_wide
    const int64_t* slots = w2slot + c.l + w2ptr[k];
    const int G = it.kind == 1 ? 1 : 32;
    for (int a = it.lane; a < d; a += G)
        for (int b = 0; b < d; ++b) kval[slots[(int64_t)a * d + b]] = (a == b) ? -1.0 : 0.0;
}

// ---------------------------------------------------------------------------
// K3: right-hand side of the z block.
//   affine:   d_s = −λ∘λ
//   combined: d_s = −λ∘λ − (W⁻¹Δs_a)∘(WΔz_a) + σμ e
//   t = λ\d_s;  rhs_z = −r_z − W t
// scratch: t1, t2 (m each).  `smu` points at σμ on the device (combined only).
// ---------------------------------------------------------------------------
__global__ void k_rhs_z(ConeView c, ConeGrid g, const double* __restrict__ lam,
                        const double* __restrict__ wbar, const double* __restrict__ eta,
                        const double* __restrict__ rz, const double* __restrict__ dsa,
                        const double* __restrict__ dza, const double* __restrict__ smu_ptr,
                        int combined, double* t, double* t1, double* t2, double* rhs) {
    ConeItem it;
    if (!cone_item(c, g, &it)) return;
    // σμ of the item's instance (per instance in a batch)
    int inst = 0;
    if (c.inst_orth) inst = it.kind == 0 ? c.inst_orth[it.idx] : c.inst_soc[it.idx];
    const double smu = combined ? smu_ptr[inst] : 0.0;
    if (it.kind == 0) {
        const int i = it.idx;
        const double li = lam[i], wi = wbar[i];
        double ds = -li * li;
        if (combined) ds += -(dsa[i] / wi) * (wi * dza[i]) + smu;
        const double ti = ds / li;
        t[i] = ti;
        rhs[i] = -rz[i] - wi * ti;
        return;
    }
    const int k = it.idx, o = c.off[k], d = c.dim[k];
    if (it.kind == 1)
        soc_rhs<1>(k, o, d, 0, c, lam, wbar, eta, rz, dsa, dza, smu, combined, t, t1, t2, rhs);
    else
        soc_rhs<32>(k, o, d, it.lane, c, lam, wbar, eta, rz, dsa, dza, smu, combined, t, t1, t2, rhs);
}

// Δs = W(t − WΔz);  scratch t1
__global__ void k_ds(ConeView c, ConeGrid g, const double* __restrict__ wbar,
                     const double* __restrict__ eta, const double* __restrict__ t,
                     const double* __restrict__ dz, double* t1, double* ds) {
    ConeItem it;
    if (!cone_item(c, g, &it)) return;
    if (it.kind == 0) {
        const int i = it.idx;
        const double wi = wbar[i];
        ds[i] = wi * (t[i] - wi * dz[i]);
        return;
    }
    const int k = it.idx, o = c.off[k], d = c.dim[k];
    const double et = eta[k];
    if (it.kind == 1) {
        soc_W<1>(o, d, 0, wbar, et, dz, t1, false);
        for (int a = 0; a < d; ++a) t1[o + a] = t[o + a] - t1[o + a];
        soc_W<1>(o, d, 0, wbar, et, t1, ds, false);
    } else {
        soc_W<32>(o, d, it.lane, wbar, et, dz, t1, false);
        __syncwarp();
        for (int a = it.lane; a < d; a += 32) t1[o + a] = t[o + a] - t1[o + a];
        __syncwarp();
        soc_W<32>(o, d, it.lane, wbar, et, t1, ds, false);
    }
}

// ---------------------------------------------------------------------------
// K4: max step (per-cone closed forms, block min → partials[block])
// Two vector pairs (u1,du1), (u2,du2) are handled in one pass (s and z).
// ---------------------------------------------------------------------------
__global__ void k_max_step(ConeView c, ConeGrid g, const double* __restrict__ u1,
                           const double* __restrict__ du1, const double* __restrict__ u2,
                           const double* __restrict__ du2, double* partial) {
    __shared__ double sm[32];
    double a = INFINITY;
    ConeItem it;
    if (cone_item(c, g, &it)) {
        if (it.kind == 0) {
            const int i = it.idx;
            if (du1[i] < 0.0) a = fmin(a, -u1[i] / du1[i]);
            if (u2 && du2[i] < 0.0) a = fmin(a, -u2[i] / du2[i]);
        } else {
            const int k = it.idx, o = c.off[k], d = c.dim[k];
            if (it.kind == 1) {
                a = soc_step<1>(o, d, 0, u1, du1);
                if (u2) a = fmin(a, soc_step<1>(o, d, 0, u2, du2));
            } else {
                a = soc_step<32>(o, d, it.lane, u1, du1);
                if (u2) a = fmin(a, soc_step<32>(o, d, it.lane, u2, du2));
            }
        }
    }
    a = warp_min_nonneg(a);  // step lengths are ≥ 0 (or +inf)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    if (wid == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sm[lane] : INFINITY;
        t = warp_min_nonneg(t);
        if (lane == 0) partial[blockIdx.x] = t;
    }
}

// initial-point shift: max over cones of (−u_i) (orthant) or (‖u_1‖ − u_0) (SOC), two vectors
__global__ void k_shift_measure(ConeView c, ConeGrid g, const double* __restrict__ u1,
                                const double* __restrict__ u2, double* partial) {
    __shared__ double sm[64];
    double m1 = -INFINITY, m2 = -INFINITY;
    ConeItem it;
    if (cone_item(c, g, &it)) {
        if (it.kind == 0) {
            m1 = -u1[it.idx];
            m2 = -u2[it.idx];
        } else {
            const int k = it.idx, o = c.off[k], d = c.dim[k];
            const int G = it.kind == 1 ? 1 : 32;
            double a1 = 0.0, a2 = 0.0;
            for (int a = 1 + it.lane; a < d; a += G) {
                a1 += u1[o + a] * u1[o + a];
                a2 += u2[o + a] * u2[o + a];
            }
            if (G == 32) { a1 = warp_sum(a1); a2 = warp_sum(a2); }
            m1 = sqrt(a1) - u1[o];
            m2 = sqrt(a2) - u2[o];
        }
    }
    m1 = -warp_min(-m1);
    m2 = -warp_min(-m2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sm[wid] = m1; sm[32 + wid] = m2; }
    __syncthreads();
    if (wid == 0) {
        const bool ok = lane < (int)(blockDim.x >> 5);
        double t1 = ok ? sm[lane] : -INFINITY, t2 = ok ? sm[32 + lane] : -INFINITY;
        t1 = -warp_min(-t1);
        t2 = -warp_min(-t2);
        if (lane == 0) { partial[2 * blockIdx.x] = t1; partial[2 * blockIdx.x + 1] = t2; }
    }
}

// u += (1 + α) e where α ≥ 0 (α read from the device; nothing when α < 0)
__global__ void k_shift_apply(ConeView c, double* u, const double* __restrict__ alpha) {
    const double a = *alpha;
    if (!(a >= 0.0)) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < c.l) u[t] += 1.0 + a;
    else if (t < c.l + c.nsoc) u[c.off[t - c.l]] += 1.0 + a;
}

// ---------------------------------------------------------------------------
// stand-alone product / division / scaling (parity entry points)
// ---------------------------------------------------------------------------
__global__ void k_prod(ConeView c, ConeGrid g, const double* u, const double* v, double* out) {
    ConeItem it;
    if (!cone_item(c, g, &it)) return;
    if (it.kind == 0) { out[it.idx] = u[it.idx] * v[it.idx]; return; }
    const int k = it.idx, o = c.off[k], d = c.dim[k];
    if (it.kind == 1) soc_prod<1>(o, d, 0, u, v, out);
    else soc_prod<32>(o, d, it.lane, u, v, out);
}
__global__ void k_div(ConeView c, ConeGrid g, const double* lam, const double* v, double* out) {
    ConeItem it;
    if (!cone_item(c, g, &it)) return;
    if (it.kind == 0) { out[it.idx] = v[it.idx] / lam[it.idx]; return; }
    const int k = it.idx, o = c.off[k], d = c.dim[k];
    if (it.kind == 1) soc_div<1>(o, d, 0, lam, v, out);
    else soc_div<32>(o, d, it.lane, lam, v, out);
}

// min over block partials → *out = min(cap, ·); one block
__global__ void k_min_partials(const double* __restrict__ partial, int n, double cap, double* out) {
    __shared__ double sm[32];
    double a = INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a = fmin(a, partial[i]);
    a = warp_min(a);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sm[wid] = a;
    __syncthreads();
    if (wid == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sm[lane] : INFINITY;
        t = warp_min(t);
        if (lane == 0) *out = fmin(t, cap);
    }
}

// ---- launchers ----------------------------------------------------------------
static int launch_w2_wide(const ConeView& c, const double* wbar, const double* eta, double* kval,
                          const int64_t* w2slot, const int64_t* w2ptr, int identity, cudaStream_t st) {
    if (!c.nwide || !kval) return 0;
    const int64_t dd = (int64_t)c.wide_maxd * c.wide_maxd;
    const dim3 grid((unsigned)((dd + 255) / 256), (unsigned)std::min(c.nwide, 65535));
    k_w2_wide<<<grid, 256, 0, st>>>(c, wbar, eta, kval, w2slot, w2ptr, identity);
    return 1;
}
int launch_nt_scaling(const ConeView& c, const double* s, const double* z, double* wbar, double* eta,
                      double* lam, double* kval, const int64_t* w2slot, const int64_t* w2ptr,
                      cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (!g.blocks()) return 0;
    k_nt_scaling<<<g.blocks(), kConeThreads, 0, st>>>(c, g, s, z, wbar, eta, lam, kval, w2slot, w2ptr);
    return 1 + launch_w2_wide(c, wbar, eta, kval, w2slot, w2ptr, 0, st);
}
int launch_w2_identity(const ConeView& c, double* kval, const int64_t* w2slot, const int64_t* w2ptr,
                       cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (!g.blocks()) return 0;
    k_w2_identity<<<g.blocks(), kConeThreads, 0, st>>>(c, g, kval, w2slot, w2ptr);
    return 1 + launch_w2_wide(c, nullptr, nullptr, kval, w2slot, w2ptr, 1, st);
}
void launch_rhs_z(const ConeView& c, const double* lam, const double* wbar, const double* eta,
                  const double* rz, const double* dsa, const double* dza, const double* smu,
                  bool combined, double* t, double* t1, double* t2, double* rhs, cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (g.blocks())
        k_rhs_z<<<g.blocks(), kConeThreads, 0, st>>>(c, g, lam, wbar, eta, rz, dsa, dza, smu,
                                                    combined ? 1 : 0, t, t1, t2, rhs);
}
void launch_ds(const ConeView& c, const double* wbar, const double* eta, const double* t,
               const double* dz, double* t1, double* ds, cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (g.blocks()) k_ds<<<g.blocks(), kConeThreads, 0, st>>>(c, g, wbar, eta, t, dz, t1, ds);
}
int max_step_partials(const ConeView& c) { return cone_grid(c).blocks(); }
void launch_max_step(const ConeView& c, const double* u1, const double* du1, const double* u2,
                     const double* du2, double cap, double* partial, double* out, cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    const int nb = g.blocks();
    if (nb) k_max_step<<<nb, kConeThreads, 0, st>>>(c, g, u1, du1, u2, du2, partial);
    k_min_partials<<<1, 256, 0, st>>>(partial, nb, cap, out);
}
void launch_shift_measure(const ConeView& c, const double* u1, const double* u2, double* partial,
                          cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (g.blocks()) k_shift_measure<<<g.blocks(), kConeThreads, 0, st>>>(c, g, u1, u2, partial);
}
void launch_shift_apply(const ConeView& c, double* u, const double* alpha, cudaStream_t st) {
    const int n = c.l + c.nsoc;
    if (n) k_shift_apply<<<(n + 255) / 256, 256, 0, st>>>(c, u, alpha);
}
void launch_prod(const ConeView& c, const double* u, const double* v, double* out, cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (g.blocks()) k_prod<<<g.blocks(), kConeThreads, 0, st>>>(c, g, u, v, out);
}
void launch_div(const ConeView& c, const double* lam, const double* v, double* out, cudaStream_t st) {
    ConeGrid g = cone_grid(c);
    if (g.blocks()) k_div<<<g.blocks(), kConeThreads, 0, st>>>(c, g, lam, v, out);
}
int cone_kernel_launches(const ConeView& c) { return cone_grid(c).blocks() ? 1 : 0; }

// ---------------------------------------------------------------------------
// Allocation-free max step.  Same kernels as launch_max_step; the block partials live
// in this fixed device array instead of caller-provided scratch.  One array per device
// (every GPU that loads the library holds it until the process exits), shared by every
// call on that device: the kernels write every slot they later read, so nothing needs
// clearing, but calls whose kernels overlap on the GPU race on it.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxPartials];

namespace {
std::mutex g_noalloc_mutex;
constexpr int kNoAllocDevices = 64;
double* g_noalloc_ptr[kNoAllocDevices] = {};
}  // namespace

// Device address of g_noalloc_partials on the current device, looked up once per device
// (the array's name in host code is only a stand-in for it).
static int noalloc_partials(double** out) {
    int dev = 0;
    QOCO_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocDevices) return QOCO_GPU_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        QOCO_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_partials));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return 0;
}

int launch_max_step_noalloc(const ConeView& c, const double* u, const double* du, double cap, double* out,
                            cudaStream_t st) {
    if (max_step_partials(c) > kNoAllocMaxPartials) return QOCO_GPU_ERR_TOO_LARGE;
    double* partial = nullptr;
    const int rc = noalloc_partials(&partial);
    if (rc) return rc;
    launch_max_step(c, u, du, nullptr, nullptr, cap, partial, out, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        // a failed launch may mean a reset context: look the address up again next time
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kNoAllocDevices) {
            std::lock_guard<std::mutex> lock(g_noalloc_mutex);
            g_noalloc_ptr[dev] = nullptr;
        }
        return cuda_fail(e, "max_step_noalloc", __FILE__, __LINE__);
    }
    return 0;
}

}  // namespace qoco
