// Device view of the supernodal structure and the per-level launch plan.
#pragma once

#include <vector>

#include "common.cuh"
#include "plan.h"

namespace qoco {


struct FactorView {
    const int* first = nullptr;      // ns: first permuted column
    const int* ncol = nullptr;       // c_s
    const int* nrow = nullptr;       // f_s
    const int64_t* row_ptr = nullptr;
    const int* rows = nullptr;       // R_s (permuted indices)
    const int64_t* front_off = nullptr;
    const int64_t* upd_off = nullptr;
    const int* rel = nullptr;
    const int* child_ptr = nullptr;
    const int* child = nullptr;
    const int64_t* amap_ptr = nullptr;
    const int64_t* amap_slot = nullptr;
    const int* amap_off = nullptr;
    const signed char* dsign = nullptr;
    const int* perm = nullptr;       // new → original
    double* front = nullptr;         // Σ f_s² doubles
    double* upd = nullptr;           // Σ r_s doubles (solve update vectors)
    double* dinv = nullptr;          // N: reciprocal pivots 1/d_j (permuted order)
    int* nreg = nullptr;             // dynamic-regularisation counter
    double eps = 1e-8, dyn_thresh = 1e-13, dyn_value = 1e-7;
};

struct FactorPlan {
    std::vector<LevelPlan> levels;
    int ntasks = 0, task_max_f = 0, task_height = 0;
    int* d_task = nullptr;   // 2·ntasks: lo, hi (inclusive) supernode ranges
    int* d_thread = nullptr; // level lists
    int* d_warp = nullptr;
    int* d_small = nullptr;
    int* d_large = nullptr;
    int* d_cta = nullptr;
};

int factor_set_attributes();
int launch_factor(const FactorPlan& P, const FactorView& a, const double* kval, cudaStream_t st);
int launch_solve(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                 double* x, bool accumulate, cudaStream_t st);

}  // namespace qoco
