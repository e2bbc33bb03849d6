// Launchers of the cone kernels (K1–K4).
#pragma once

#include "cones.cuh"

namespace qoco {

// Both return the number of kernels launched.
int launch_nt_scaling(const ConeView& c, const double* s, const double* z, double* wbar, double* eta,
                      double* lam, double* kval, const int64_t* w2slot, const int64_t* w2ptr,
                      cudaStream_t st);
int launch_w2_identity(const ConeView& c, double* kval, const int64_t* w2slot, const int64_t* w2ptr,
                       cudaStream_t st);
void launch_rhs_z(const ConeView& c, const double* lam, const double* wbar, const double* eta,
                  const double* rz, const double* dsa, const double* dza, const double* smu,
                  bool combined, double* t, double* t1, double* t2, double* rhs, cudaStream_t st);
void launch_ds(const ConeView& c, const double* wbar, const double* eta, const double* t,
               const double* dz, double* t1, double* ds, cudaStream_t st);
int max_step_partials(const ConeView& c);
// min(cap, max step of (u1,du1) and, if u2 != NULL, (u2,du2)) → *out (device)
void launch_max_step(const ConeView& c, const double* u1, const double* du1, const double* u2,
                     const double* du2, double cap, double* partial, double* out, cudaStream_t st);
void launch_shift_measure(const ConeView& c, const double* u1, const double* u2, double* partial,
                          cudaStream_t st);
void launch_shift_apply(const ConeView& c, double* u, const double* alpha, cudaStream_t st);
void launch_prod(const ConeView& c, const double* u, const double* v, double* out, cudaStream_t st);

// Block partials the allocation-free max step can hold (one per block of the cone grid:
// ⌈l/256⌉ + ⌈#SOC ≤ 32/256⌉ + ⌈#SOC > 32/8⌉); 8192 doubles = 64 KiB per device.
constexpr int kNoAllocMaxPartials = 8192;
// Max step with the partials in a fixed device array (no allocation); returns 0 or a
// QOCO_GPU_ERR_* code (TOO_LARGE when the cone grid needs more than kNoAllocMaxPartials).
int launch_max_step_noalloc(const ConeView& c, const double* u, const double* du, double cap, double* out,
                            cudaStream_t st);
void launch_div(const ConeView& c, const double* lam, const double* v, double* out, cudaStream_t st);

}  // namespace qoco
