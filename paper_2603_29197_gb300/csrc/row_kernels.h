// Row kernels over the KKT value array and the interior-point scalars they feed.
#pragma once

#include "common.cuh"

namespace qoco {

// Full symmetric KKT in CSR (original x | y | z order); val is the one value array
// that the −W² update writes into and that the factor assembly and SpMV read.
struct KKTView {
    int N = 0, n = 0, p = 0, m = 0;
    const int64_t* rowptr = nullptr;
    const int* colidx = nullptr;
    const double* val = nullptr;
    // rows with more than kLongRow entries (the dense rows of a factor model or a budget
    // constraint): the row kernels skip them and one block per listed row takes them
    const int* long_rows = nullptr;
    int n_long = 0;
};
constexpr int kLongRow = 2048;

// Device-resident scalars of one solve (read back to the host once per iteration).
struct IPMScalars {
    // residual pass
    double pobj, dobj, gap, mu;
    double rx_inf, ry_inf, rz_inf, Px_inf, Aty_inf, Gtz_inf, Ax_inf, Gx_inf, s_inf;
    int converged, converged_inacc, nonfinite, max_iters;  // max_iters: batched solves
    // constants set at setup
    double c_inf, b_inf, h_inf, nu;
    double abstol, reltol, abstol_inacc, reltol_inacc;
    double refine_tol, step_fraction;
    // steps
    double alpha_a, sigma, sigma_mu, alpha, alpha_max;
    double shift[2];
    // refinement
    double normK, berr;
    double refine_den;        // ‖K‖∞‖x‖∞ + ‖r‖∞ of the last refinement residual (berr's denominator)
    double berr_cw;           // componentwise backward error max_i |r − Kx|_i / (|K||x| + |r|)_i
    int refine_done, pad1;
    // shared state of the dataflow kernels: two spare words, the timeout flag, the
    // work-item counter (zeroed together before each solve)
    unsigned int bar_count, bar_gen;
    int bar_err;
    unsigned int sched_next;
};

constexpr int kResNSum = 5;
constexpr int kResNV = 14;

// Size (doubles) of the per-block partial buffer the row kernels need for any LPR.
int row_partials(int N, int n_long);
// Each launcher returns −1 without launching when `cap` (the partial buffer's size in
// doubles) is too small for its grid, else the number of kernels it launched.
int launch_residual(const KKTView& K, int lpr, const double* xyz, const double* s, const double* c,
                    const double* b, const double* h, double* r, double* partial, int64_t cap,
                    IPMScalars* S, cudaStream_t st);
// cw: also the componentwise backward error (IPMScalars::berr_cw; 0 otherwise) and, when
// den is given (N doubles), (|K||x| + |r|)_i per row
int launch_spmv_res(const KKTView& K, int lpr, const double* x, const double* r, double* res,
                    double* partial, int64_t cap, IPMScalars* S, cudaStream_t st, bool cw = false,
                    double* den = nullptr);
int launch_norm_inf(const KKTView& K, int lpr, double* partial, int64_t cap, IPMScalars* S,
                    cudaStream_t st);

}  // namespace qoco
