// Launch plan of the supernodal factorisation and solves (host side, plain C++).
#pragma once

#include <vector>

#include "symbolic.h"

namespace qoco {

constexpr int kSmemFront = 160;       // fronts up to this order are factored in shared memory
constexpr int kMaxSolveFront = 26000; // solve kernels keep one front vector in shared memory
constexpr int kMaxFactorFront = 5600;  // CTA factor keeps a 4-column panel + signs in shared memory
constexpr int kThreadFront = 8;     // fronts up to this order are handled by one thread
constexpr int kWarpFront = 48;      // fronts up to this order are handled by one warp
constexpr int kPairFront = 28;      // dataflow factorisation: two such fronts share a warp
constexpr int kWarpsPerBlock = 4;    // warps per block of the warp-level kernels
constexpr int kWideLevel = 2432;     // levels with at least this many fronts (16 per SM) use warps
// Fronts at least this large are factored and solved by grid-wide kernel sequences
// (panels of kBigNB columns), one front after the other, when their level holds at most
// kBigPerLevel of them; fronts of at least kHugeFront always are.
constexpr int kBigFront = 160;
constexpr int kHugeFront = 1024;
constexpr int kBigPerLevel = 64;
constexpr int kBigNB = 64;
constexpr int kGroupTile = 16;  // tile of a leaf group's split-K rank-K product

// Launch plan of one factorisation / solve: the supernodes of each tree level, fronts
// up to kThreadFront by one thread each (so that every FP64 warp instruction serves 32
// fronts), up to kWarpFront by one warp each, up to kSmemFront by a CTA in shared
// memory, larger ones by a CTA in global memory or by the large-front kernels.
struct LevelPlan {
    // factorisation lists
    int n_thread = 0, off_thread = 0;
    int n_warp = 0, off_warp = 0, max_warp_f = 0;
    int n_small = 0, off_small = 0, max_small = 0;
    int n_large = 0, off_large = 0, max_large_f = 0;
    // solve lists (by front order only: a solve front's dependent chain is short)
    int n_sthread = 0, off_sthread = 0;
    int n_swarp = 0, off_swarp = 0, max_swarp_f = 0;
    int n_cta = 0, off_cta = 0, max_cta_f = 0;
    // large fronts (factor and solves): big[off_big .. off_big + n_big)
    int n_big = 0, off_big = 0;
};

// Host-side lists from which the device plan is uploaded.
struct PlanHost {
    std::vector<LevelPlan> levels;
    std::vector<int> thread, warp, small, large;        // factorisation
    std::vector<int> sthread, swarp, cta;               // solves
    std::vector<int> big;                               // large fronts (factor and solves)
    // dataflow solve: work items in topological (level) order; item ≥ 0 is a warp
    // front, item < 0 is the batch −(item+1) of ≤ 32 one-thread fronts
    // (sthread[tb_ptr[b] .. tb_ptr[b+1]))
    std::vector<int> items, tb_ptr;
    // dataflow factorisation items (kind in the low two bits, see factor.cu):
    // batches of ≤ 128 one-thread fronts (thread[ftb_ptr[b] ..]), groups of ≤ 4 warp
    // fronts (warp[fwg_ptr[g] ..]) and single CTA fronts
    std::vector<int> fitems, ftb_ptr, fwg_ptr;
    int max_f = 0;
};

// Builds the plan: per-level lists of every supernode and the dataflow item lists.
void build_plan(const Symbolic& S, PlanHost* P);

}  // namespace qoco
