// Launch plan of the supernodal factorisation and solves: per-level lists and dataflow items.
#include "plan.h"

#include <algorithm>
#include <numeric>

namespace qoco {

void build_plan(const Symbolic& S, PlanHost* P) {
    const int ns = S.ns;
    *P = PlanHost();
    std::vector<int> f(S.sn_nrow), lev(S.level);
    for (int s = 0; s < ns; ++s) P->max_f = std::max(P->max_f, f[s]);
    // supernodes by level
    P->levels.assign(S.n_levels, LevelPlan());
    std::vector<std::vector<int>> byl(S.n_levels);
    for (int s = 0; s < ns; ++s)
        byl[lev[s]].push_back(s);
    for (int l = 0; l < S.n_levels; ++l) {
        LevelPlan& L = P->levels[l];
        // fronts sorted by decreasing order so that the lanes of a one-thread-per-front
        // warp run similar trip counts
        std::stable_sort(byl[l].begin(), byl[l].end(), [&](int x, int y) { return f[x] > f[y]; });
        L.off_thread = (int)P->thread.size();
        L.off_warp = (int)P->warp.size();
        L.off_small = (int)P->small.size();
        L.off_large = (int)P->large.size();
        L.off_sthread = (int)P->sthread.size();
        L.off_swarp = (int)P->swarp.size();
        L.off_cta = (int)P->cta.size();
        L.off_big = (int)P->big.size();
        // A level with few fronts cannot fill the GPU with one warp per front, and each
        // warp would walk its front's long dependent FP64 chain alone: in the
        // factorisation such levels get a CTA per front (its threads split every
        // update).  Wide levels keep one warp (or one thread) per front for throughput.
        int nmid = 0, nbig = 0;
        for (int s : byl[l]) {
            nmid += f[s] > kThreadFront;
            nbig += f[s] >= kBigFront;
        }
        const bool wide = nmid >= kWideLevel;
        for (int s : byl[l]) {
            if (f[s] >= kHugeFront || (f[s] >= kBigFront && nbig <= kBigPerLevel)) {
                P->big.push_back(s);
                continue;
            }
            if (f[s] <= kThreadFront && (wide || nmid == 0)) {
                P->thread.push_back(s);
            } else if (f[s] <= kWarpFront && wide) {
                P->warp.push_back(s);
                L.max_warp_f = std::max(L.max_warp_f, f[s]);
            } else if (f[s] <= kSmemFront) {
                P->small.push_back(s);
                L.max_small = std::max(L.max_small, f[s]);
            } else {
                P->large.push_back(s);
                L.max_large_f = std::max(L.max_large_f, f[s]);
            }
            if (f[s] <= kThreadFront) {
                P->sthread.push_back(s);
            } else if (f[s] <= kWarpFront) {
                P->swarp.push_back(s);
                L.max_swarp_f = std::max(L.max_swarp_f, f[s]);
            } else {
                P->cta.push_back(s);
                L.max_cta_f = std::max(L.max_cta_f, f[s]);
            }
        }
        L.n_thread = (int)P->thread.size() - L.off_thread;
        L.n_warp = (int)P->warp.size() - L.off_warp;
        L.n_small = (int)P->small.size() - L.off_small;
        L.n_large = (int)P->large.size() - L.off_large;
        L.n_sthread = (int)P->sthread.size() - L.off_sthread;
        L.n_swarp = (int)P->swarp.size() - L.off_swarp;
        L.n_cta = (int)P->cta.size() - L.off_cta;
        L.n_big = (int)P->big.size() - L.off_big;
    }
    // dataflow items, level by level: batches of 32 one-thread fronts, then warp fronts.
    // The one-thread fronts of consecutive levels are contiguous in sthread, so batch b
    // covers sthread[tb_ptr[b] .. tb_ptr[b+1]).
    P->tb_ptr.assign(1, 0);
    for (int l = 0; l < (int)P->levels.size(); ++l) {
        const LevelPlan& L = P->levels[l];
        for (int t = 0; t < L.n_sthread; t += 32) {
            const int b = (int)P->tb_ptr.size() - 1;  // its start tb_ptr[b] = off_sthread + t
            P->tb_ptr.push_back(L.off_sthread + std::min(t + 32, L.n_sthread));
            P->items.push_back(-(b + 1));
        }
        for (int t = 0; t < L.n_swarp; ++t) P->items.push_back(P->swarp[L.off_swarp + t]);
    }
    // dataflow factorisation items, level by level
    P->ftb_ptr.assign(1, 0);
    P->fwg_ptr.assign(1, 0);
    for (int l = 0; l < (int)P->levels.size(); ++l) {
        const LevelPlan& L = P->levels[l];
        for (int t = 0; t < L.n_thread; t += 128) {
            const int b = (int)P->ftb_ptr.size() - 1;
            P->ftb_ptr.push_back(L.off_thread + std::min(t + 128, L.n_thread));
            P->fitems.push_back((b << 2) | 0);
        }
        // the level's warp fronts come in decreasing order: groups of 4 (one warp each),
        // then, from the first of order ≤ kPairFront, groups of 8 (two per warp, neighbours
        // in that order pairing fronts of about the same size)
        int npair0 = L.n_warp;
        for (int t = 0; t < L.n_warp; ++t)
            if (P->warp[L.off_warp + t] >= 0 && f[P->warp[L.off_warp + t]] <= kPairFront) { npair0 = t; break; }
        for (int t = 0; t < npair0; t += 4) {
            const int g = (int)P->fwg_ptr.size() - 1;
            P->fwg_ptr.push_back(L.off_warp + std::min(t + 4, npair0));
            P->fitems.push_back((g << 2) | 1);
        }
        for (int t = npair0; t < L.n_warp; t += 8) {
            const int g = (int)P->fwg_ptr.size() - 1;
            P->fwg_ptr.push_back(L.off_warp + std::min(t + 8, L.n_warp));
            P->fitems.push_back((g << 2) | 3);
        }
        for (int t = 0; t < L.n_small; ++t) P->fitems.push_back((P->small[L.off_small + t] << 2) | 2);
    }
    // drop empty trailing levels
    while (!P->levels.empty() &&
           P->levels.back().n_sthread + P->levels.back().n_swarp + P->levels.back().n_cta +
                   P->levels.back().n_big == 0)
        P->levels.pop_back();
}

}  // namespace qoco
