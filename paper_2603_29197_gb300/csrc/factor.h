// Device view of the supernodal structure and the per-level launch plan.
#pragma once

#include <vector>

#include "common.cuh"
#include "plan.h"

namespace qoco {


// One child edge of the supernodal tree, in the parent's child order: where the child's
// update block starts in the front array (its trailing r×r block, leading dimension
// fc), and where its relative indices / solve update vector start (upd_off).
struct ChildInfo {
    int64_t u_off;
    int64_t rel_off;
    int fc;
    int r;
};

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
    const ChildInfo* cinfo = nullptr;  // parallel to child
    const int64_t* amap_ptr = nullptr;
    const int64_t* amap_slot = nullptr;
    const int64_t* amap_off = nullptr;  // col·f + row (64-bit: large fronts exceed 2^31 entries)
    const signed char* dsign = nullptr;
    const int* perm = nullptr;       // new → original
    const int* parent = nullptr;     // supernodal tree parent (−1 for roots)
    double* front = nullptr;         // Σ f_s² doubles
    double* upd = nullptr;           // Σ r_s doubles (solve update vectors)
    double* dinv = nullptr;          // N: reciprocal pivots 1/d_j (permuted order)
    int* nreg = nullptr;             // dynamic-regularisation counter
    // per supernode: 1 = factored by the leaf-group kernel (a one-level leaf whose update
    // reaches its large parent through the group's rank-K product), skipped elsewhere
    const signed char* skip = nullptr;
    double eps = 1e-8, dyn_thresh = 1e-13, dyn_value = 1e-7;
    double eps32 = 0.0;  // sign-aware shift of the scaled FP32 large fronts' diagonal
    // scaled FP32 large fronts: the smallest accepted signed pivot (one device double, raised
    // by the host after a breakdown) and the breakdown flag the writeback sets when the
    // factor holds a non-finite or overgrown entry
    const double* piv32 = nullptr;
    int* bad32 = nullptr;
};

struct FactorPlan {
    std::vector<LevelPlan> levels;
    int* d_thread = nullptr; // level lists
    int* d_warp = nullptr;
    int* d_small = nullptr;
    int* d_large = nullptr;
    int* d_cta = nullptr;
    int* d_sthread = nullptr;
    int* d_swarp = nullptr;
    // dataflow solve (items in topological order, see PlanHost)
    bool dataflow = false;
    int nitems = 0, dataflow_grid = 0, dataflow_fmax = 0;
    int* d_items = nullptr;
    int* d_tb_ptr = nullptr;
    int* d_fdone = nullptr;  // per supernode: epoch of its finished forward step
    int* d_bdone = nullptr;  // per supernode: epoch of its finished backward step
    // dataflow factorisation
    bool fdataflow = false;
    int nfitems = 0, fdataflow_grid = 0, fdataflow_fmax = 0;
    int* d_fitems = nullptr;
    int* d_ftb_ptr = nullptr;
    int* d_fwg_ptr = nullptr;
    int* d_cdone = nullptr;  // per supernode: epoch of its finished factorisation
    // batches of independent instances: one CTA takes one whole instance at a time from a
    // queue (largest instances first) and runs its factorisation / solve level by level
    // with block barriers.  Two schedules (fronts of order ≤ kThreadFront one per thread,
    // or every front one warp), each runnable with 4 or 8 warps per CTA: candidates 1–4.
    struct InstSched {
        int* d_lv_ptr = nullptr;  // ninst + 1: the instance's level entries
        int* d_ent = nullptr;     // 3 per entry: thread fronts [t0, w0), warp fronts [w0, end) of sched
        int* d_sched = nullptr;
    };
    bool inst = false;
    int ninst = 0, inst_fmax = 0, inst_variant = 0;
    int inst_fgrid[2] = {0, 0}, inst_sgrid[2] = {0, 0};  // persistent grids for 4 / 8 warps
    int* d_inst_order = nullptr;
    InstSched isched[2];
    unsigned int* d_inst_next = nullptr;
    // large fronts (grid-wide kernel sequences, bigfront.cu); host lists indexed by the
    // levels' off_big/n_big
    std::vector<int> big_s, big_f, big_c;
    std::vector<int64_t> big_front_off, big_amap_n;
    // per large front, for each of its f rows p: the child entries (child edge index into
    // FactorView::cinfo, position in that child's update rows) that land on row p, in
    // child order: segment ea_ptr[big_ea_off[idx] + p .. + p + 1) of ea_child / ea_pos
    std::vector<int64_t> big_ea_off;
    // inverses of the 64×64 unit-lower diagonal blocks of each large front (row-major,
    // block b of front idx at big_linv + big_linv_off[idx] + b·64·64), written during the
    // factorisation (used there for the panel's rows below, and by the solves)
    std::vector<int64_t> big_linv_off;
    double* big_linv = nullptr;
    // leaf groups: many childless children of one large front with the same update rows
    // (an arrowhead border).  Their pivots are factored one warp per member; the parent
    // receives −Σ L21·D·L21ᵀ as one split-K rank-K product instead of one update matrix
    // per member.  Host lists; per group: parent's index into big_*, members, r, K.
    struct LeafGroup {
        int big_idx = 0;
        int r = 0;                 // update rows (common to the members)
        int K = 0;                 // member columns with entries in the update rows
        int nmem = 0;
        int64_t rel_off = 0;       // one member's relative indices (all equal)
        int* d_members = nullptr;  // member supernodes
        int* d_gmem = nullptr;     // K: member (index into d_members) of each gathered column
        int* d_gloc = nullptr;     // K: its column inside the member front
        int64_t* d_updoff = nullptr;  // each member's update vector in FactorView::upd
    };
    std::vector<LeafGroup> groups;
    double* grp_L = nullptr;       // K × r (column k of L21ᵀ contiguous) of the group being assembled
    double* grp_W = nullptr;       // K × r: (L21·D)ᵀ
    double* grp_part = nullptr;    // split-K partial tiles (also the solve's member-sum partials)
    int grp_split = 0;
    int64_t* d_ea_ptr = nullptr;
    int* d_ea_child = nullptr;
    int* d_ea_pos = nullptr;
    int max_big_f = 0;
    bool big_fp32 = false;         // factor large fronts in FP32 (mixed precision)
    float* big_work32 = nullptr;   // max_big_f² FP32 working front
    // FP32 fronts: TF32 head / remainder of the outer panel's L and W rows (Lhi, Llo, Whi,
    // Wlo, each max_big_f × 4·kBigNB row-major) and their TMA tensor maps (opaque bytes)
    float* big_split = nullptr;
    double* big_scale = nullptr;   // max_big_f: symmetric scaling of the FP32 front being factored
    alignas(64) unsigned char big_tmaps[4 * 128] = {};
    void* big_w = nullptr;         // max_big_f × 4·kBigNB doubles: panel rows W (FP64), or W and L (FP32)
    double* big_v = nullptr;       // max_big_f solve work vector
    double* big_y = nullptr;       // max_big_f solved block values
    // dataflow solves of the large fronts: block counter and per-block flags (reset before
    // each launch), the solver's error flag and its poll bound
    int* big_ctl = nullptr;
    int* df_err = nullptr;
    long long df_spins = 0;
};

// Shared state of one dataflow solve launch.
struct DataflowState {
    unsigned int* next;  // work-item counter (zeroed before each launch)
    int* err;            // set when a dependency wait ran out of polls
    int epoch;           // flag value that marks "done in this launch"
    long long max_spins;
};

int factor_set_attributes();
// Per-instance kernels of a batch: grid sizes for the fronts' largest order fmax (≤ kWarpFront).
int plan_instances(FactorPlan& P, int fmax);
int launch_inst_factor(const FactorPlan& P, const FactorView& a, const double* kval, int variant, cudaStream_t st);
int launch_inst_solve(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                      double* x, bool accumulate, int variant, cudaStream_t st);
// Launches a probe whose dataflow wait is on a flag nothing publishes; returns
// QOCO_GPU_ERR_DEVICE_TIMEOUT when the bounded wait ran out as designed.
int selftest_wait_timeout(long long max_spins, cudaStream_t st);
int plan_dataflow_solve(FactorPlan& P, int max_warp_f, bool any_cta_front);
int plan_dataflow_factor(FactorPlan& P, int fmax, bool any_large);
// The forward solve of one right-hand side fused into the dataflow factorisation: each
// front runs its forward step (L u = b restricted to the front, w = D⁻¹u, its update
// vector for the parent) right after its own factorisation, with the factor still on
// chip, and publishes its factor and forward flags together.  rhs == nullptr: no fusion.
struct FwdFuse {
    const double* rhs = nullptr;
    double* w = nullptr;
    int* fdone = nullptr;  // the solve's forward flags
    int epoch = 0;         // the solve epoch the backward launch will use
};
int launch_factor_dataflow(const FactorPlan& P, const FactorView& a, const double* kval, const DataflowState& ds,
                           cudaStream_t st, const FwdFuse& fz = FwdFuse());
// bwd_only: the backward sweep alone, after a factorisation that fused the forward one
int launch_solve_dataflow(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                          double* x, bool accumulate, const DataflowState& ds, cudaStream_t st,
                          bool bwd_only = false);
int launch_factor(const FactorPlan& P, const FactorView& a, const double* kval, cudaStream_t st);
// One large front (P.big_*[idx]): partial LDLᵀ, or the forward / backward solve step.
int big_set_attributes();
// The leaf-group members' pivot columns (all groups), one warp per member.
int launch_leaf_groups(const FactorPlan& P, const FactorView& a, const double* kval, cudaStream_t st);
// Encodes the tensor maps of big_split (mixed precision).
int big_tma_setup(FactorPlan& P);
int launch_big_factor(const FactorPlan& P, const FactorView& a, const double* kval, int idx, cudaStream_t st);
int launch_big_fwd(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, int idx,
                   cudaStream_t st);
int launch_big_bwd(const FactorPlan& P, const FactorView& a, const double* w, double* xp, double* x,
                   bool accumulate, int idx, cudaStream_t st);
int launch_solve(const FactorPlan& P, const FactorView& a, const double* rhs, double* w, double* xp,
                 double* x, bool accumulate, cudaStream_t st);

}  // namespace qoco
