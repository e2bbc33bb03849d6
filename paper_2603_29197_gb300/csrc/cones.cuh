// Cone kernels (paper §2.1 "cone operations", §2.3 one worker per cone).
//
// K = R^l_+ × Q^{q_0} × …: orthant entries get one thread each; a second-order cone
// of dimension ≤ kSmallCone gets one thread; a larger one gets one warp whose lanes
// stride over the block and combine partial dot products with shuffles.  Every
// kernel launch covers all three groups through one grid (blocks [0,b_orth) for the
// orthant, then the small cones, then the large cones, 8 warps per block).
#pragma once

#include "common.cuh"

namespace qoco {

struct ConeView {
    int l = 0, nsoc = 0, m = 0;
    const int* off = nullptr;    // nsoc: start of each SOC block inside the m-vector
    const int* dim = nullptr;    // nsoc
    const int* small = nullptr;  // ids of SOCs with dim ≤ kSmallCone
    const int* large = nullptr;  // ids of SOCs with dim > kSmallCone
    int nsmall = 0, nlarge = 0;
    // SOCs with dim > kWideCone: their dim² block of −W² is written by a grid-wide kernel
    // (one thread per entry) instead of the cone's warp
    const int* wide = nullptr;
    int nwide = 0, wide_maxd = 0;
    // batched problems: instance of each orthant entry (l) and of each SOC (nsoc); null
    // for a single problem (everything is instance 0)
    const int* inst_orth = nullptr;
    const int* inst_soc = nullptr;
};

constexpr int kConeThreads = 256;
constexpr int kWideCone = 64;

struct ConeGrid {
    int b_orth = 0, b_small = 0, b_large = 0;
    int blocks() const { return b_orth + b_small + b_large; }
};
inline ConeGrid cone_grid(const ConeView& c) {
    ConeGrid g;
    g.b_orth = (c.l + kConeThreads - 1) / kConeThreads;
    g.b_small = (c.nsmall + kConeThreads - 1) / kConeThreads;
    g.b_large = (c.nlarge + kConeThreads / kWarp - 1) / (kConeThreads / kWarp);
    return g;
}

// Work item of the calling thread: kind 0 orthant index i, kind 1 small cone k
// (lane 0 of a group of 1), kind 2 large cone k (lane 0..31).  Returns false when idle.
struct ConeItem {
    int kind, idx, lane;
};
__device__ __forceinline__ bool cone_item(const ConeView& c, const ConeGrid& g, ConeItem* it) {
    int b = blockIdx.x;
    if (b < g.b_orth) {
        it->kind = 0;
        it->idx = b * kConeThreads + threadIdx.x;
        it->lane = 0;
        return it->idx < c.l;
    }
    b -= g.b_orth;
    if (b < g.b_small) {
        int t = b * kConeThreads + threadIdx.x;
        it->kind = 1;
        it->lane = 0;
        if (t >= c.nsmall) return false;
        it->idx = c.small[t];
        return true;
    }
    b -= g.b_small;
    int w = b * (kConeThreads / kWarp) + (threadIdx.x >> 5);
    it->kind = 2;
    it->lane = threadIdx.x & 31;
    if (w >= c.nlarge) return false;
    it->idx = c.large[w];
    return true;
}

template <int G>
__device__ __forceinline__ double gsum(double v) {
    if constexpr (G == 1) return v;
    else return group_sum<G>(v);
}
template <int G>
__device__ __forceinline__ void gsync() {
    if constexpr (G > 1) __syncwarp();
}

// ---- per-SOC building blocks (group of G lanes, lane in [0,G)) -------------------

// out = u∘v = (uᵀv, u_0 v_1 + v_0 u_1)
template <int G>
__device__ __forceinline__ void soc_prod(int o, int d, int lane, const double* u, const double* v,
                                         double* out) {
    const double u0 = u[o], v0 = v[o];
    double dot = 0.0;
    for (int a = lane; a < d; a += G) dot += u[o + a] * v[o + a];
    dot = gsum<G>(dot);
    gsync<G>();
    for (int a = 1 + lane; a < d; a += G) out[o + a] = u0 * v[o + a] + v0 * u[o + a];
    if (lane == 0) out[o] = dot;
}

// out = λ\v: w_0 = (λ_0 v_0 − λ_1ᵀv_1)/((λ_0 − ‖λ_1‖)(λ_0 + ‖λ_1‖)), w_1 = (v_1 − w_0 λ_1)/λ_0
template <int G>
__device__ __forceinline__ void soc_div(int o, int d, int lane, const double* lam, const double* v,
                                        double* out) {
    const double l0 = lam[o], v0 = v[o];
    double lv = 0.0, ll = 0.0;
    for (int a = 1 + lane; a < d; a += G) {
        lv += lam[o + a] * v[o + a];
        ll += lam[o + a] * lam[o + a];
    }
    lv = gsum<G>(lv);
    ll = gsum<G>(ll);
    const double nl = sqrt(ll);
    const double w0 = (l0 * v0 - lv) / ((l0 - nl) * (l0 + nl));
    gsync<G>();
    for (int a = 1 + lane; a < d; a += G) out[o + a] = (v[o + a] - w0 * lam[o + a]) / l0;
    if (lane == 0) out[o] = w0;
}

// out = W v (inv = false) or W⁻¹ v (inv = true) with
// W = η [[w̄_0, w̄_1ᵀ], [w̄_1, I + w̄_1 w̄_1ᵀ/(1 + w̄_0)]], W⁻¹ = η⁻¹ [[w̄_0, −w̄_1ᵀ], [−w̄_1, I + w̄_1 w̄_1ᵀ/(1 + w̄_0)]]
template <int G>
__device__ __forceinline__ void soc_W(int o, int d, int lane, const double* wbar, double eta,
                                      const double* v, double* out, bool inv) {
    const double w0 = wbar[o], v0 = v[o];
    double wv = 0.0;
    for (int a = 1 + lane; a < d; a += G) wv += wbar[o + a] * v[o + a];
    wv = gsum<G>(wv);
    gsync<G>();
    if (!inv) {
        const double coef = v0 + wv / (1.0 + w0);
        for (int a = 1 + lane; a < d; a += G) out[o + a] = eta * (v[o + a] + coef * wbar[o + a]);
        if (lane == 0) out[o] = eta * (w0 * v0 + wv);
    } else {
        const double coef = -v0 + wv / (1.0 + w0);
        const double ie = 1.0 / eta;
        for (int a = 1 + lane; a < d; a += G) out[o + a] = ie * (v[o + a] + coef * wbar[o + a]);
        if (lane == 0) out[o] = ie * (w0 * v0 - wv);
    }
}

// NT scaling of one SOC block (s̄ = s/√(sᵀJs), z̄ = z/√(zᵀJz), γ = √((1 + s̄ᵀz̄)/2),
// w̄ = (s̄ + J z̄)/(2γ), η = (sᵀJs/zᵀJz)^{1/4}, λ = W z); optionally writes −W² − 0 into
// the d·d KKT value slots of the block (W² = η²(2 w̄ w̄ᵀ − J)).
template <int G>
__device__ __forceinline__ void soc_nt(int k, int o, int d, int lane, const double* s, const double* z,
                                       double* wbar, double* eta, double* lam, double* kval,
                                       const int64_t* slots) {
    const double s0 = s[o], z0 = z[o];
    double ss = 0.0, zz = 0.0, sz = 0.0;
    for (int a = 1 + lane; a < d; a += G) {
        const double sa = s[o + a], za = z[o + a];
        ss += sa * sa;
        zz += za * za;
        sz += sa * za;
    }
    ss = gsum<G>(ss);
    zz = gsum<G>(zz);
    sz = gsum<G>(sz);
    const double ns1 = sqrt(ss), nz1 = sqrt(zz);
    const double sj = (s0 - ns1) * (s0 + ns1);
    const double zj = (z0 - nz1) * (z0 + nz1);
    const double rs = sqrt(sj), rz = sqrt(zj);
    const double dotbar = (s0 * z0 + sz) / (rs * rz);
    const double gam = sqrt(0.5 * (1.0 + dotbar));
    const double inv2g = 0.5 / gam;
    const double w0 = (s0 / rs + z0 / rz) * inv2g;
    const double et = sqrt(sqrt(sj / zj));
    double wz = 0.0;
    for (int a = 1 + lane; a < d; a += G) {
        const double wa = (s[o + a] / rs - z[o + a] / rz) * inv2g;
        wbar[o + a] = wa;
        wz += wa * z[o + a];
    }
    wz = gsum<G>(wz);
    const double coef = z0 + wz / (1.0 + w0);
    for (int a = 1 + lane; a < d; a += G) lam[o + a] = et * (z[o + a] + coef * wbar[o + a]);
    if (lane == 0) {
        wbar[o] = w0;
        eta[k] = et;
        lam[o] = et * (w0 * z0 + wz);
    }
    if (kval) {
        gsync<G>();
        const double e2 = et * et;
        for (int a = lane; a < d; a += G) {
            const double wa = wbar[o + a];
            for (int b = 0; b < d; ++b) {
                const double J = (a == b) ? (a == 0 ? 1.0 : -1.0) : 0.0;
                kval[slots[(int64_t)a * d + b]] = -e2 * (2.0 * wa * wbar[o + b] - J);
            }
        }
    }
}

// sup{α ≥ 0 : u + α du ∈ Q} from a = du_0² − ‖du_1‖², b = u_0 du_0 − u_1ᵀdu_1,
// c = u_0² − ‖u_1‖² > 0: the smallest positive root of aα² + 2bα + c (inf if none).
__device__ __forceinline__ double soc_root(double a, double b, double c) {
    if (!(c > 0.0)) return 0.0;
    if (a == 0.0) return b < 0.0 ? -c / (2.0 * b) : INFINITY;
    const double disc = b * b - a * c;
    if (disc < 0.0) return INFINITY;
    const double sq = sqrt(disc);
    if (a < 0.0) {
        // roots of opposite sign
        return b >= 0.0 ? -(b + sq) / a : c / (sq - b);
    }
    if (b >= 0.0) return INFINITY;
    return c / (sq - b);  // smaller of the two positive roots
}

template <int G>
__device__ __forceinline__ double soc_step(int o, int d, int lane, const double* u, const double* du) {
    double uu = 0.0, dd = 0.0, ud = 0.0;
    for (int a = 1 + lane; a < d; a += G) {
        const double ua = u[o + a], da = du[o + a];
        uu += ua * ua;
        dd += da * da;
        ud += ua * da;
    }
    uu = gsum<G>(uu);
    dd = gsum<G>(dd);
    ud = gsum<G>(ud);
    const double u0 = u[o], d0 = du[o];
    const double nu1 = sqrt(uu), nd1 = sqrt(dd);
    const double a = (d0 - nd1) * (d0 + nd1);
    const double b = u0 * d0 - ud;
    const double c = (u0 - nu1) * (u0 + nu1);
    return soc_root(a, b, c);
}

// Right-hand side of one SOC block of the z rows (see k_rhs_z): d_s = −λ∘λ (affine) or
// −λ∘λ − (W⁻¹Δs_a)∘(WΔz_a) + σμ e (combined), t = λ\d_s, rhs_z = −r_z − W t.
template <int G>
__device__ __forceinline__ void soc_rhs(int k, int o, int d, int lane, const ConeView& c, const double* lam,
                        const double* wbar, const double* eta, const double* rz, const double* dsa,
                        const double* dza, double smu, bool combined, double* t, double* t1,
                        double* t2, double* rhs) {
    const double et = eta[k];
    soc_prod<G>(o, d, lane, lam, lam, t1);  // t1 = λ∘λ
    gsync<G>();
    if (combined) {
        soc_W<G>(o, d, lane, wbar, et, dsa, t2, true);   // t2 = W⁻¹Δs_a
        soc_W<G>(o, d, lane, wbar, et, dza, t, false);   // t  = WΔz_a
        gsync<G>();
        // t1 += t2∘t
        double dot = 0.0;
        for (int a = lane; a < d; a += G) dot += t2[o + a] * t[o + a];
        dot = gsum<G>(dot);
        const double a0 = t2[o], b0 = t[o];
        gsync<G>();
        for (int a = 1 + lane; a < d; a += G) t1[o + a] += a0 * t[o + a] + b0 * t2[o + a];
        if (lane == 0) t1[o] += dot;
        gsync<G>();
    }
    // t1 = d_s = −t1 + σμ e
    for (int a = lane; a < d; a += G) t1[o + a] = -t1[o + a] + ((a == 0 && combined) ? smu : 0.0);
    gsync<G>();
    soc_div<G>(o, d, lane, lam, t1, t);  // t = λ\d_s
    gsync<G>();
    soc_W<G>(o, d, lane, wbar, et, t, t2, false);  // t2 = W t
    gsync<G>();
    for (int a = lane; a < d; a += G) rhs[o + a] = -rz[o + a] - t2[o + a];
}

}  // namespace qoco
