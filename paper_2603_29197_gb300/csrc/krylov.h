// FP64 vector kernels of the GMRES refinement (GMRES-IR: restarted GMRES on the KKT
// matrix K, row-scaled and right-preconditioned by the LDLᵀ factor, used when plain
// refinement with a factor that has FP32 large fronts does not reach its target).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace qoco {

constexpr int kKrylovRestart = 30;  // basis vectors per GMRES cycle

// Doubles of scratch the dot kernels need (block partials for up to kKrylovRestart + 2
// vectors at once).
int krylov_partials();
// out[k] = V_kᵀw (or out[k] += …) for the nv vectors V_k = V + k·ld, fixed-order sums.
int launch_dots(const double* V, int64_t ld, int nv, const double* w, int64_t N, double* partial, double* out,
                bool accumulate, cudaStream_t st);
// w −= Σ c[k]·V_k (c: nv device scalars)
int launch_sub_combination(const double* V, int64_t ld, int nv, const double* c, double* w, int64_t N,
                           cudaStream_t st);
// u = Σ c[k]·V_k
int launch_combination(const double* V, int64_t ld, int nv, const double* c, double* u, int64_t N,
                       cudaStream_t st);
// dst = sign·src / √(*nrm2) (nrm2: one device scalar)
int launch_scale_by_norm(const double* src, double* dst, int64_t N, const double* nrm2, double sign,
                         cudaStream_t st);

// dst = D·src (inverse = false) or D⁻¹·src (inverse = true) for D = diag(1/den), the row
// scaling of the GMRES refinement (den_i = (|K||x| + |r|)_i; 1 where not positive)
int launch_row_scale(const double* src, const double* den, double* dst, int64_t N, bool inverse, cudaStream_t st);

}  // namespace qoco
