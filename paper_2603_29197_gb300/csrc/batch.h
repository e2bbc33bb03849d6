// Per-instance scalars of a batch of independent problems solved as one block-diagonal
// stack (see batch.cu).  Layout of the stack: instance b's x entries are
// [xo[b], xo[b+1]), its y entries [yo[b], yo[b+1]); the stacked cone has every
// instance's orthant rows first (instance b: [lo[b], lo[b+1])) and then every instance's
// second-order cones (instance b: cones [ko[b], ko[b+1]), their rows L + [so[b], so[b+1])
// where L is the stacked orthant dimension).
#pragma once

#include <cuda_runtime.h>

#include "cones.cuh"
#include "row_kernels.h"

namespace qoco {

struct BatchView {
    int nb = 0;
    const int *xo = nullptr, *yo = nullptr, *lo = nullptr, *ko = nullptr, *so = nullptr;
    const int* inst_row = nullptr;  // N: instance of each KKT row
    const double *nu = nullptr, *c_inf = nullptr, *b_inf = nullptr, *h_inf = nullptr;
    double *pobj = nullptr, *dobj = nullptr, *gap = nullptr, *mu = nullptr;
    double* res = nullptr;  // 3 per instance: ‖r_x‖∞, ‖r_y‖∞, ‖r_z‖∞
    double *alpha_max = nullptr, *sigma_mu = nullptr, *alpha = nullptr;
    int *conv = nullptr, *conv_inacc = nullptr, *nonfinite = nullptr, *iters = nullptr;
};

// Each launcher returns the number of kernels it launched.
int launch_batch_residual(const KKTView& K, const BatchView& B, int L, const double* xyz, const double* s,
                          const double* c, const double* b, const double* h, double* r, double* aux, int iter,
                          const IPMScalars& tol, IPMScalars* S, cudaStream_t st);
// per-instance min step of (u1, du1), (u2, du2) → B.alpha_max; items: l + nsoc doubles
int launch_batch_max_step(const ConeView& c, const BatchView& B, const double* u1, const double* du1,
                          const double* u2, const double* du2, double* items, cudaStream_t st);
// initial-point shift of s and z per instance; items: 2(l + nsoc), shift2: 2·nb doubles
int launch_batch_shift(const ConeView& c, const BatchView& B, double* s, double* z, double* items,
                       double* shift2, cudaStream_t st);
int launch_batch_sigma(const BatchView& B, cudaStream_t st);
int launch_batch_step(const BatchView& B, double step_fraction, double* xyz, double* s, const double* d,
                      const double* ds, int N, int nzoff, int m, cudaStream_t st);

}  // namespace qoco
