// The batched interior-point solve as one persistent launch (batch_ipm.cu).
#pragma once

#include "batch.h"
#include "cones.cuh"
#include "factor.h"
#include "row_kernels.h"

namespace qoco {

struct BatchIPMArgs {
    KKTView K;      // stacked KKT (full symmetric CSR, original order)
    ConeView C;     // stacked cones (offsets and dimensions of every SOC)
    FactorView F;   // supernodal structure and front storage of the stack
    BatchView B;    // per-instance offsets, constants and results
    int L = 0;      // stacked orthant dimension
    // per-instance level schedule of the instance's supernodes (FactorPlan::InstSched)
    const int* lv_ptr = nullptr;
    const int* ent = nullptr;
    const int* sched = nullptr;
    const int* order = nullptr;  // instances, largest first
    unsigned int* next = nullptr;
    const int64_t* w2slot = nullptr;
    const int64_t* w2ptr = nullptr;
    double* kval = nullptr;  // KKT values (the −W² slots are written)
    const double *c = nullptr, *b = nullptr, *h = nullptr;
    double *xyz = nullptr, *s = nullptr;
    double *d_aff = nullptr, *ds_aff = nullptr, *d_cmb = nullptr, *ds_cmb = nullptr, *r = nullptr,
           *rhs = nullptr, *wbar = nullptr, *eta = nullptr, *lam = nullptr, *t = nullptr, *t1 = nullptr,
           *t2 = nullptr, *sol_w = nullptr, *sol_xp = nullptr, *res = nullptr;
    double abstol = 0, reltol = 0, abstol_inacc = 0, reltol_inacc = 0, refine_tol = 0, step_fraction = 0;
    int max_iter = 0, max_refine = 0, fmax = 1;
    bool mixed = false;  // FP32 fronts, FP64 refinement, FP64 refactor of an instance on a miss
};

// Grid of the persistent kernel with nw ∈ {1, 2, 4} warps per CTA, compiled for 16 (dense
// = 0) or 32 (dense = 1) resident warps per SM, for fronts of order ≤ fmax (0 when it cannot
// run); sets the kernel's shared-memory attribute.
int batch_ipm_grid(int nw, int dense, bool mixed, int fmax, int nb, int* grid);
// One launch solving every instance (results in B: conv, conv_inacc, nonfinite, iters,
// pobj, dobj, gap); resets the queue counter first.
int launch_batch_ipm(const BatchIPMArgs& A, int nw, int dense, int grid, cudaStream_t st);
// Every-instance summary into S (converged, converged_inacc, nonfinite, max_iters, gap).
int launch_batch_summary(const BatchView& B, IPMScalars* S, cudaStream_t st);

}  // namespace qoco
