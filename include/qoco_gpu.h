/*
 * qoco_gpu.h — C ABI of a GB300 (sm_103a) interior-point solver for
 *
 *     minimise ½xᵀPx + cᵀx   subject to   Gx ⪯_K h,  Ax = b            (paper §1, eq. (1))
 *
 * with K = R^l_+ × Q^{q_1} × … × Q^{q_nsoc} (non-negative orthant times second-order
 * cones).  The call sequence follows the paper's interface (§2.1, Listing 1:
 * setup(n, m, p, P, c, A, b, G, h, l, nsoc, q) then solve()).  One iteration factors
 * the quasidefinite KKT matrix of eq. (2) once and solves with it twice (§2.2); the
 * factorisation, the solves and the cone operations (§2.1, §2.3) all run in this
 * library's own CUDA kernels; data cross host→device once at setup and device→host
 * once at the end (§2.3).
 *
 * Conventions shared by every entry point
 *   - Matrices are CSC, 0-based, row indices strictly increasing within a column,
 *     no duplicates.  P holds the upper triangle (diagonal included) of a symmetric
 *     PSD matrix (§3 sizes problems by "the upper half of P").
 *   - G's rows are ordered: the l orthant rows first, then the SOC blocks in the
 *     order of q; so m = l + Σ q[k].  A vector u is in Q^q when u_0 ≥ ‖u_{1:q}‖.
 *   - Pointers documented "host" are read (or written) during the call only; the
 *     caller keeps ownership.  Pointers documented "device" must be CUDA device
 *     memory of the current device, 8-byte aligned.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Calls taking a stream are ordered on it and return before the GPU
 *     work finishes unless stated otherwise.
 *   - Return value: 0 (or a positive non-error status) on success, a negative
 *     QOCO_GPU_ERR_* code on failure.  No global error state is kept; the solver's
 *     info struct carries a message for the last failure.
 */
#ifndef QOCO_GPU_H
#define QOCO_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define QOCO_GPU_SOLVED               0  /* stopping tests met at abstol/reltol          */
#define QOCO_GPU_SOLVED_INACCURATE    1  /* max_iter reached, met the *_inacc tolerances  */
#define QOCO_GPU_MAX_ITER             2  /* max_iter reached                               */
#define QOCO_GPU_ERR_INVALID_DIMS    -1
#define QOCO_GPU_ERR_INVALID_CSC     -2  /* unsorted / duplicate / out-of-range / P not upper */
#define QOCO_GPU_ERR_INVALID_CONE    -3  /* l < 0, nsoc < 0, some q < 2, l + Σq ≠ m       */
#define QOCO_GPU_ERR_NONFINITE_DATA  -4
#define QOCO_GPU_ERR_NUMERICAL       -5  /* NaN/Inf in an iterate, or an iterate left the cone */
#define QOCO_GPU_ERR_OOM             -6
#define QOCO_GPU_ERR_CUDA            -7
#define QOCO_GPU_ERR_DEVICE_TIMEOUT  -8  /* a bounded device wait (dataflow dependency flag) ran out */
#define QOCO_GPU_ERR_NO_FACTOR       -9  /* a call needs a factorisation that does not exist */
#define QOCO_GPU_ERR_INVALID_ARG    -10
#define QOCO_GPU_ERR_NOT_IMPLEMENTED -11
#define QOCO_GPU_ERR_TOO_LARGE      -12  /* exceeds a fixed-size buffer of an allocation-free entry point */

/* ---- orderings for the symbolic analysis ---------------------------------- */
#define QOCO_GPU_ORDER_AUTO     0  /* the cheaper of AMD and ND by the analysis' cost model */
#define QOCO_GPU_ORDER_AMD      1  /* approximate minimum degree                           */
#define QOCO_GPU_ORDER_ND       2  /* nested dissection, AMD inside the leaves             */
#define QOCO_GPU_ORDER_NATURAL  3  /* identity (x, then y, then z)                         */

typedef struct {
    int n_rows, n_cols, nnz;
    const int* colptr;     /* host, n_cols + 1 */
    const int* rowidx;     /* host, nnz        */
    const double* val;     /* host, nnz        */
} qoco_csc;

/* Settings.  The paper fixes only the tolerances (ε_abs = ε_rel = 1e-7, §3); every
 * other default is a documented reading of the method the paper defers to. */
typedef struct {
    double abstol, reltol;              /* 1e-7, 1e-7 */
    double abstol_inacc, reltol_inacc;  /* 1e-5, 1e-5 */
    int max_iter;                       /* 200 */
    double static_reg;                  /* ε: +ε on the x block, −ε on y and z (1e-8) */
    double dyn_reg_thresh;              /* pivot with sign·d < thresh ... (1e-13) */
    double dyn_reg_value;               /* ... is replaced by sign·value (1e-7) */
    int max_refine;                     /* iterative-refinement steps per solve (10) */
    double refine_tol;                  /* normwise backward-error target (1e-10) */
    double step_fraction;               /* 0.99 */
    int ordering;                       /* QOCO_GPU_ORDER_* (AUTO) */
    int nd_leaf;                        /* ND stops splitting below this many nodes; 0:
                                           automatic, N_K/2048 clamped to 64..256 (0) */
    int64_t wait_polls;                 /* polls (each sleeps ~32–64 ns) a device-side dependency
                                           wait of the dataflow factor/solve kernels may take
                                           before it gives up and the call returns
                                           QOCO_GPU_ERR_DEVICE_TIMEOUT; ≤ 0 = 20000000, about a
                                           second (default 0) */
    int verbose;                        /* 0: silent; 1: one line per iteration on stdout;
                                           2: also one line per refinement of a solve */
    int mixed_precision;                /* 1: fronts of order ≥ 160 factored in FP32 (scaled
                                           symmetrically so that each row's largest entry is
                                           1, FP32 accumulation, trailing updates on the tensor
                                           cores as three TF32 products, pivots below a floor
                                           replaced by ± the floor), solves and refinement in
                                           FP64; an
                                           FP32 factor that breaks down (a non-finite entry or
                                           one above 1e30) is redone with a ten times larger
                                           floor (1e-5 at the start of a solve, at most 1e-2);
                                           a solve whose plain
                                           refinement stalls or misses refine_tol within
                                           max_refine steps goes on with restarted GMRES on K,
                                           row-scaled and preconditioned by the factor (≤ 3
                                           cycles of 30, fewer when an FP64 refactor would cost
                                           less than the iterations); on an FP32 factor a solve
                                           must meet refine_tol both normwise and componentwise
                                           (max_i |r − Kx|_i / (|K||x| + |r|)_i); if that
                                           misses too, it refactors in FP64; the next
                                           iteration factors in FP32 again unless the last two
                                           FP32 factorisations failed.  Batches on the
                                           persistent kernel factor every front in FP32 and
                                           refactor an instance in FP64 when its refinement
                                           misses (default 0) */
    double mixed_reg;                   /* mixed precision: δ added to the diagonal of each
                                           scaled FP32 front (row maxima 1), with the pivot's
                                           sign (+ on x rows, − on y and z rows): a quasidefinite
                                           shift that bounds the FP32 elimination's growth; the
                                           refinement against the unregularised K removes it
                                           (default 0) */
    int batch_schedule;                 /* schedule of a batch (qoco_gpu_setup_batch) whose
                                           fronts all fit one warp: 0 or 6 = one persistent
                                           kernel per batched solve, each CTA running whole
                                           instances' interior-point iterations on chip (its
                                           tile configuration — warps per CTA, registers per
                                           thread — timed on the whole batch at the first
                                           solve, a search over 3–4 of the 6 tiles that
                                           halves the warps per CTA while that pays); 1–5 = the
                                           host-driven iteration loop with per-instance factor
                                           and solve kernels, one CTA per instance at a time
                                           (1: 4 warps per CTA, fronts of order ≤ 8 one per
                                           thread; 2: 8 warps, same split; 3: 4 warps, every
                                           front one warp; 4: 8 warps, every front one warp)
                                           or (5) the shared kernels of single problems;
                                           7–12 = the persistent kernel with a fixed tile
                                           instead of the tuning (7, 8: 1 warp per CTA; 9,
                                           10: 2 warps; 11, 12: 4 warps; odd: 16 resident
                                           warps per SM, even: 32), tuned all the same when
                                           the batch cannot launch that tile (default 0).
                                           Other batches always use 5. */
} qoco_gpu_settings;

typedef struct {
    int status;                 /* last solve's status code */
    int iters;
    double pobj, dobj, gap, pres, dres;
    double setup_time_s;        /* whole qoco_gpu_setup call (host wall clock) */
    double analysis_time_s;     /* ordering + symbolic factorisation (host) */
    double solve_time_s;        /* last qoco_gpu_solve, host wall clock incl. its sync */
    int64_t kkt_dim;            /* N_K = n + p + m */
    int64_t kkt_nnz;            /* stored entries of the full symmetric KKT */
    int64_t l_nnz;              /* entries of L below the diagonal (algorithmic, no amalgamation zeros) */
    int64_t front_entries;      /* Σ f_s², the dense front storage in doubles */
    double factor_flops;        /* Σ_j (c_j² + 2 c_j), c_j = below-diagonal count of L's column j */
    int n_supernodes, n_levels, max_front;
    int ordering_used;
    int refine_steps;           /* refinement steps taken during the last solve */
    double last_backward_error;
    int64_t kernel_launches;    /* this library's kernel launches during the last solve */
    int64_t h2d_bytes;          /* host→device bytes copied by setup */
    int64_t d2h_bytes;          /* device→host bytes read back during the last solve */
    int large_fronts;           /* fronts factored by the grid-wide large-front kernels */
    int fp32_factors;           /* factorisations of the last solve with FP32 large fronts */
    int fp64_escalations;       /* refinements that missed the target on an FP32 factor */
    int batch_schedule_used;    /* batches: the schedule in use (1–6 as in the settings) */
    int krylov_steps;           /* GMRES iterations of the last solve (refinement of solves
                                   whose factor has FP32 large fronts, see mixed_precision) */
    int batch_warps;            /* batches on the persistent kernel, as chosen by its tuning:   */
    int batch_thread_fronts;    /* warps per CTA, whether fronts of order ≤ 8 get one thread, */
    int batch_warps_per_sm;     /* and the resident warps per SM it was compiled for (16, 32)  */
    int fp32_floor_raises;      /* FP32 factorisations of the last solve that broke down and were
                                   redone in FP32 with a ten times larger pivot floor */
    char message[160];
} qoco_gpu_info;

/* Per-phase device time of the solves run while profiling is on (CUDA events recorded
 * on the solver's stream around each phase; milliseconds summed over launches). */
#define QOCO_GPU_PHASE_FACTOR  0   /* numeric LDLᵀ: every level launch of one factorisation */
#define QOCO_GPU_PHASE_SOLVE   1   /* one forward + backward triangular solve */
#define QOCO_GPU_PHASE_CONE    2   /* one cone kernel (scaling, rhs, Δs, step) */
#define QOCO_GPU_PHASE_ROW     3   /* one residual / SpMV / norm pass */
#define QOCO_GPU_NPHASE        4
typedef struct {
    double ms[QOCO_GPU_NPHASE];
    int64_t calls[QOCO_GPU_NPHASE];
    int64_t launches[QOCO_GPU_NPHASE];  /* kernel launches inside the timed phases */
} qoco_gpu_profile;

typedef struct qoco_gpu_solver qoco_gpu_solver;
typedef struct qoco_gpu_cones qoco_gpu_cones;

/* Fills `s` with the defaults listed in qoco_gpu_settings. */
void qoco_gpu_default_settings(qoco_gpu_settings* s);

/* ---- solver --------------------------------------------------------------- */

/* Validates the data, assembles the KKT pattern of eq. (2) (with every diagonal
 * slot present and the SOC blocks of −WᵀW dense), orders it, runs the symbolic
 * supernodal analysis on the host, and copies everything to the current device
 * (paper §2.3: copy once at setup).  P may be NULL (P = 0); A and b may be NULL
 * when p = 0; q may be NULL when nsoc = 0; settings NULL = defaults.
 * On success *out owns all device memory of the solver.  On failure *out is NULL
 * and nothing is leaked.  Errors: INVALID_DIMS, INVALID_CSC, INVALID_CONE,
 * NONFINITE_DATA, OOM, CUDA. */
int qoco_gpu_setup(qoco_gpu_solver** out, int n, int m, int p,
                   const qoco_csc* P, const double* c,
                   const qoco_csc* A, const double* b,
                   const qoco_csc* G, const double* h,
                   int l, int nsoc, const int* q,
                   const qoco_gpu_settings* settings);

/* Runs the predictor–corrector interior-point loop on the GPU from a fresh initial
 * point until the stopping tests hold or max_iter is reached (paper §2: one
 * factorisation and two solves per iteration).  Blocks until the solve ends (one
 * 64-byte device→host read per iteration carries the stopping test).  Returns the
 * solve status (SOLVED, SOLVED_INACCURATE, MAX_ITER) or an error (NUMERICAL, CUDA,
 * DEVICE_TIMEOUT: one of the dataflow kernels' bounded waits gave up, the solve stops). */
int qoco_gpu_solve(qoco_gpu_solver* solver, void* stream);

/* Copies the last iterate to host buffers (any may be NULL): x[n], s[m], y[p], z[m];
 * info (may be NULL) receives the statistics.  Synchronises the solver's stream. */
int qoco_gpu_get_solution(const qoco_gpu_solver* solver, double* x, double* s,
                          double* y, double* z, qoco_gpu_info* info);

/* Device pointers of the solver-owned iterate (valid until cleanup): x[n], s[m], y[p], z[m]. */
int qoco_gpu_solution_device(const qoco_gpu_solver* solver, const double** x,
                             const double** s, const double** y, const double** z);

/* ---- batches of independent problems ------------------------------------------ */

/* Sets up `batch` independent instances of eq. (1) (paper §1) as one solver: the
 * instances are stacked block-diagonally and solved by one interior-point loop whose
 * scalars — residual norms, gap, μ, step lengths, σ, the stopping test — are kept per
 * instance; an instance that meets the stopping test takes zero steps from then on, and
 * the loop ends when every instance has (or at max_iter).  One factorisation and two
 * solves per iteration serve the whole batch (the KKT matrix of eq. (2) is block
 * diagonal, its supernodal tree a forest).  The paper solves one problem at a time;
 * this is one of the forms grown beyond it.
 *
 * With ordering AUTO the cost model counts the batch's independent trees (their
 * dependent chains of fronts overlap), and the factor/solve schedule is picked by
 * timing at the first factorisation unless settings->batch_schedule fixes it.
 *
 * Arrays of length `batch` (host): n, m, p, l, nsoc; P, A, G are arrays of `batch` CSC
 * matrices (P[i] with colptr == NULL means P_i = 0; A[i] is ignored when p[i] = 0);
 * c, b, h, q are arrays of `batch` host pointers (b[i] may be NULL when p[i] = 0).
 * Each instance follows the conventions above (orthant rows first in its G).  Layout of
 * the stacked iterate returned by qoco_gpu_get_solution: see qoco_gpu_batch_offsets.
 * Errors: as qoco_gpu_setup (the message names the failing instance);
 * NOT_IMPLEMENTED when an instance has no cone row (m = 0: its barrier parameter
 * ν = l + nsoc would be zero). */
int qoco_gpu_setup_batch(qoco_gpu_solver** out, int batch, const int* n, const int* m,
                         const int* p, const qoco_csc* P, const double* const* c,
                         const qoco_csc* A, const double* const* b, const qoco_csc* G,
                         const double* const* h, const int* l, const int* nsoc,
                         const int* const* q, const qoco_gpu_settings* settings);

/* Number of instances (0 for a solver made by qoco_gpu_setup). */
int qoco_gpu_batch_size(const qoco_gpu_solver* solver);

/* Offsets (host arrays of batch + 1 ints, any may be NULL) of the stacked iterate:
 * instance i's x is x[xo[i] .. xo[i+1]), its y is y[yo[i] .. yo[i+1]); its s and z
 * are the orthant part [lo[i], lo[i+1]) followed by the SOC part L + [so[i], so[i+1])
 * with L = lo[batch]; its cones are ko[i] .. ko[i+1]. */
int qoco_gpu_batch_offsets(const qoco_gpu_solver* solver, int* xo, int* yo, int* lo, int* ko,
                           int* so);

/* Per-instance results of the last solve (host arrays of length batch, any may be NULL):
 * status (QOCO_GPU_SOLVED, _SOLVED_INACCURATE, _MAX_ITER or _ERR_NUMERICAL), the
 * iteration at which the instance met the stopping test, primal and dual objective,
 * and sᵀz.  Synchronises the device. */
int qoco_gpu_batch_info(const qoco_gpu_solver* solver, int* status, int* iters, double* pobj,
                        double* dobj, double* gap);

/* Copies the solver's iterate into caller DEVICE buffers x[n], s[m], y[p], z[m] (any may
 * be NULL), ordered on `stream` (device-to-device copies, no host round trip). */
int qoco_gpu_copy_solution(const qoco_gpu_solver* solver, double* x, double* s, double* y,
                           double* z, void* stream);

/* Statistics of setup and of the last solve. */
int qoco_gpu_get_info(const qoco_gpu_solver* solver, qoco_gpu_info* info);

/* Adjoint of the solution map (not in the paper; one of the forms grown beyond the
 * plain solver): implicit differentiation of the optimality conditions of eq. (1) at
 * the final iterate (x, s, y, z) of the last qoco_gpu_solve,
 *
 *     Px + c + Aᵀy + Gᵀz = 0,   Ax = b,   Gx + s = h,   s ∘ z = (final value),
 *
 * with the complementarity linearised exactly in the cone's Jordan algebra,
 * z ∘ ds + s ∘ dz = 0, i.e. ds = −Arw(z)⁻¹Arw(s) dz (for the orthant ds = −(s/z) dz).
 * For g = ∂L/∂(x, y, z) it solves K̂ᵀv = g, where K̂ is eq. (2)'s matrix with that
 * block in place of −WᵀW, by iterative refinement preconditioned with the final LDLᵀ
 * factor (reused; the NT scaling of the iterate before the last step); if the
 * refinement stalls, it refactors once at the final iterate's NT scaling.  Then
 *
 *     dc = −v_x,  db = v_y,  dh = v_z,
 *     dA_rc = −(y_r v_x,c + v_y,r x_c),  dG_rc = −(z_r v_x,c + v_z,r x_c),
 *     dP_ij = −(v_x,i x_j + v_x,j x_i) for a stored upper entry i < j,  dP_ii = −v_x,i x_i.
 *
 * All pointers are DEVICE memory of the solver's device.  dx[n], dy[p], dz[m] are the
 * incoming gradients (NULL = zero); outputs (NULL = not wanted): dP_val[nnz(P)] on P's
 * stored upper pattern in CSC order, dc[n], dA_val[nnz(A)], db[p], dG_val[nnz(G)],
 * dh[m].  Synchronous (the refinement reads its backward error on the host).  The
 * derivative exists where the solution is strictly complementary; on degenerate
 * solutions the refinement may not converge and QOCO_GPU_ERR_NUMERICAL is returned.
 * The call overwrites the −WᵀW slots of the solver's KKT values and its work vectors
 * (the next qoco_gpu_solve starts from its own initial point, so it is unaffected).
 * Errors: NO_FACTOR (no completed solve), NUMERICAL, CUDA, DEVICE_TIMEOUT. */
int qoco_gpu_backward(qoco_gpu_solver* solver, const double* dx, const double* dy,
                      const double* dz, double* dP_val, double* dc, double* dA_val,
                      double* db, double* dG_val, double* dh, void* stream);

/* Refinement statistics of the last qoco_gpu_backward: steps taken, final normwise
 * backward error of K̂ᵀv = g, and whether it refactored (host outputs, may be NULL). */
int qoco_gpu_backward_info(const qoco_gpu_solver* solver, int* refine_steps,
                           double* backward_error, int* refactored);

/* Parametric re-solve (paper §3.2 names set-up as QOCO-GPU's bottleneck; this keeps
 * the ordering, symbolic analysis and every device buffer): replaces the values of the
 * problem data without changing any sparsity pattern.  P_val[nnz(P)], A_val[nnz(A)],
 * G_val[nnz(G)] follow the CSC order given at setup; c[n], b[p], h[m]; NULL keeps the
 * current values.  on_device = 0: host pointers, checked for finiteness
 * (NONFINITE_DATA); on_device = 1: device pointers, not checked (a non-finite value
 * surfaces as NUMERICAL in the next solve).  Ordered on `stream`; the next
 * qoco_gpu_solve starts from a fresh initial point. */
int qoco_gpu_update_data(qoco_gpu_solver* solver, const double* P_val, const double* c,
                         const double* A_val, const double* b, const double* G_val,
                         const double* h, int on_device, void* stream);

/* Turns per-phase CUDA-event timing on (1: every phase; 2: the factorisation phase alone,
 * two events per factorisation, the lightest timing of the dominant kernel) or off (0)
 * and clears the totals.  Other values: QOCO_GPU_ERR_INVALID_ARG. */
int qoco_gpu_set_profiling(qoco_gpu_solver* solver, int on);
/* Reads the per-phase totals accumulated since profiling was turned on. */
int qoco_gpu_get_profile(const qoco_gpu_solver* solver, qoco_gpu_profile* out);

/* Releases every resource of the solver (NULL is accepted). */
int qoco_gpu_cleanup(qoco_gpu_solver* solver);

/* ---- KKT system at a caller-chosen iterate (shared-iterate parity) ---------- */

/* Sets the scaling from interior points s, z (device, m each): NT scaling of every
 * cone (§2.1 "Nesterov-Todd scalings"), writes −W² into the KKT value array through
 * the index map, and refactors K_ε (§2.2, once per iteration).  Synchronous. */
int qoco_gpu_kkt_factor_at(qoco_gpu_solver* solver, const double* s, const double* z,
                           void* stream);

/* Solves K x = r with the current factorisation plus iterative refinement against the
 * unregularised K (device r, x of length N_K in the original x, y, z order).
 * Synchronous; *refine_steps and *backward_error (host, may be NULL) report the
 * refinement.  Errors: NO_FACTOR. */
int qoco_gpu_kkt_solve(qoco_gpu_solver* solver, const double* r, double* x,
                       int* refine_steps, double* backward_error, void* stream);

/* Copies the current full symmetric KKT (original order, CSR) to host buffers:
 * rowptr[N_K+1], colidx[kkt_nnz], val[kkt_nnz] (any may be NULL). */
int qoco_gpu_get_kkt(const qoco_gpu_solver* solver, int64_t* rowptr, int* colidx, double* val);

/* Copies the current factor as dense arrays (host), for N_K ≤ 4096 only:
 * perm[N_K] (new → original index), L[N_K·N_K] row-major unit lower triangular in the
 * permuted order, D[N_K].  Errors: INVALID_ARG (too large), NO_FACTOR. */
int qoco_gpu_get_factor_dense(const qoco_gpu_solver* solver, int* perm, double* L, double* D);

/* Copies the reciprocal pivots 1/d_j that the factorisation stored for the solves
 * (host dinv[N_K], permuted order; computed on the device by two Newton–Raphson steps
 * from the hardware's approximate reciprocal).  Errors: NO_FACTOR. */
int qoco_gpu_get_pivot_reciprocals(const qoco_gpu_solver* solver, double* dinv);

/* Failure-detection self-test of the dependency wait used by the dataflow factorisation
 * and solve kernels (the paper has no counterpart): launches a probe whose wait is on a
 * flag that nothing ever publishes, so the wait runs out after max_polls polls (≥ 1,
 * ~32–64 ns each), raises the error flag and returns instead of hanging.  Returns
 * QOCO_GPU_ERR_DEVICE_TIMEOUT when that happened (the expected outcome), 0 if the wait
 * ended otherwise, INVALID_ARG for max_polls < 1, or a CUDA error.  Synchronous; the
 * context stays usable. */
int qoco_gpu_selftest_wait_timeout(long long max_polls, void* stream);

/* FP64 throughput of the current device, measured by this library's own kernels (the
 * paper has no counterpart; these are the FP64 roofline denominators of the factor
 * kernels, §2.2): every warp of 8 blocks per SM issues long runs of independent FP64
 * FMAs (dfma_gflops) or of FP64 tensor-core products mma.sync m8n8k4 (dmma_gflops);
 * best of five timed launches (CUDA events on `stream`), GFLOP/s counting 2 flops per
 * FMA and 512 per m8n8k4 product.  Host outputs.  Synchronous; allocates a few KB. */
int qoco_gpu_fp64_peaks(double* dfma_gflops, double* dmma_gflops, void* stream);

/* ---- stand-alone cone kernels (paper §2.1, §2.3) ---------------------------- */

/* Creates a device descriptor of K = R^l_+ × Q^{q_0} × …; q host, nsoc entries ≥ 2. */
int qoco_gpu_cones_create(qoco_gpu_cones** out, int l, int nsoc, const int* q);
int qoco_gpu_cones_destroy(qoco_gpu_cones* cones);

/* NT scaling of interior s, z (device, m each).  Outputs (device): w[m] (orthant:
 * √(s_i/z_i); SOC block: w̄), eta[nsoc], lambda[m] = W z. */
int qoco_gpu_cone_nt_scaling(const qoco_gpu_cones* cones, const double* s, const double* z,
                             double* w, double* eta, double* lambda, void* stream);

/* Jordan product out = u∘v and division out = λ\v (device vectors of length m). */
int qoco_gpu_cone_product(const qoco_gpu_cones* cones, const double* u, const double* v,
                          double* out, void* stream);
int qoco_gpu_cone_division(const qoco_gpu_cones* cones, const double* lam, const double* v,
                           double* out, void* stream);

/* Largest α with u + α du ∈ K (u interior), capped at `cap` (pass +inf for none):
 * per-cone closed forms and a min over cones.  Writes one double to alpha (device).
 * `scratch` (device) must hold qoco_gpu_cone_max_step_scratch_bytes(cones) bytes. */
size_t qoco_gpu_cone_max_step_scratch_bytes(const qoco_gpu_cones* cones);
int qoco_gpu_cone_max_step(const qoco_gpu_cones* cones, const double* u, const double* du,
                           double cap, double* alpha, void* scratch, void* stream);

/* Allocation-free variant of qoco_gpu_cone_max_step (the paper has no counterpart):
 * for callers that must not allocate device memory while they run — code that is being
 * captured into a CUDA graph, real-time control loops that reserve all memory up front,
 * or hosts whose allocator is owned by another framework — this call takes no scratch
 * argument and calls no cudaMalloc, cudaFree or allocating library routine.  Its block
 * partials live in one fixed 64 KiB device array (8192 doubles) that every GPU loading
 * the library holds until the process exits.
 *   - Same inputs, output and result as qoco_gpu_cone_max_step (the cones descriptor is
 *     created beforehand by qoco_gpu_cones_create).
 *   - Returns QOCO_GPU_ERR_TOO_LARGE, without launching, when the cone grid needs more
 *     than 8192 partials (⌈l/256⌉ + ⌈#SOC of dim ≤ 32 / 256⌉ + ⌈#SOC of dim > 32 / 8⌉).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture.  The address is kept for the life of the process: it assumes the
 *     device's context is not reset (cudaDeviceReset) in between; a call whose launch
 *     fails forgets it, so the call after that looks it up again.
 *   - All calls on a device share the array; every slot a call reads is written earlier
 *     in the same call, so nothing carries over, but calls whose kernels overlap on the
 *     GPU (different streams, or threads) race on it and must be serialised. */
int qoco_gpu_cone_max_step_noalloc(const qoco_gpu_cones* cones, const double* u, const double* du,
                                   double cap, double* alpha, void* stream);

/* ---- host-only analysis (no GPU needed) ---------------------------------------- */

/* Runs the same validation, KKT assembly, ordering and symbolic analysis as
 * qoco_gpu_setup on the host only and reports their statistics in *info; perm
 * (host, N_K, may be NULL) receives the final new → original ordering.
 * sn_ptr (host, may be NULL) receives the first permuted column of each supernode
 * followed by N_K (n_supernodes + 1 entries; call once with NULL to learn the count);
 * sn_nrow and sn_level (host, n_supernodes entries each, may be NULL) receive each
 * supernode's front order f_s and its height in the supernodal tree.
 * Errors as for setup. */
int qoco_gpu_analyze(int n, int m, int p, const qoco_csc* P, const qoco_csc* A,
                     const qoco_csc* G, int l, int nsoc, const int* q,
                     const qoco_gpu_settings* settings, qoco_gpu_info* info, int* perm,
                     int* sn_ptr, int* sn_nrow, int* sn_level);

/* The analysis qoco_gpu_setup_batch makes, on the host only (arguments as there, without
 * the vectors c, b, h): the instances are validated and stacked block-diagonally, each
 * distinct instance pattern (sizes, cone dimensions, P, A and G sparsity) is ordered and
 * analysed once (paper §2.2: the analysis runs once per sparsity pattern) and the stack's
 * KKT pattern and supernodal analysis are assembled from those; with the natural ordering
 * the stack is analysed as one problem.  Outputs as for qoco_gpu_analyze, in the stack's
 * numbering (x of every instance, then y, then every orthant row, then every SOC row).
 * Errors as for qoco_gpu_setup_batch. */
int qoco_gpu_analyze_batch(int batch, const int* n, const int* m, const int* p,
                           const qoco_csc* P, const qoco_csc* A, const qoco_csc* G,
                           const int* l, const int* nsoc, const int* const* q,
                           const qoco_gpu_settings* settings, qoco_gpu_info* info, int* perm,
                           int* sn_ptr, int* sn_nrow, int* sn_level);

#ifdef __cplusplus
}
#endif
#endif /* QOCO_GPU_H */
