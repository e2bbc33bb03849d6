// Launch plan of the supernodal factorisation: subtree tasks + level lists.
#include "plan.h"

#include <algorithm>
#include <numeric>

namespace qoco {

void build_plan(const Symbolic& S, bool allow_tasks, int target_tasks, PlanHost* P) {
    const int ns = S.ns;
    *P = PlanHost();
    std::vector<int> f(S.sn_nrow), par(S.sn_parent), lev(S.level);
    for (int s = 0; s < ns; ++s) P->max_f = std::max(P->max_f, f[s]);
    // a subtree is eligible when every front in it is small; it is usable as a task only
    // when its supernodes form a contiguous index range (true for postordered trees)
    std::vector<char> elig(ns, 0);
    std::vector<int> fd(ns), size(ns, 1);
    for (int s = 0; s < ns; ++s) { elig[s] = f[s] <= kWarpFront; fd[s] = s; }
    for (int s = 0; s < ns; ++s) {
        const int p = par[s];
        if (p < 0) continue;
        if (!elig[s]) elig[p] = 0;
        fd[p] = std::min(fd[p], fd[s]);
        size[p] += size[s];
    }
    std::vector<char> contiguous(ns);
    for (int s = 0; s < ns; ++s) contiguous[s] = size[s] == s - fd[s] + 1;
    auto is_root = [&](int s, int H) {
        if (!elig[s] || !contiguous[s] || lev[s] >= H) return false;
        const int p = par[s];
        return p < 0 || !elig[p] || !contiguous[p] || lev[p] >= H;
    };
    int H = 0;
    if (allow_tasks && ns > 0) {
        int best_h = 0, best_n = 0;
        for (int h = 1; h <= S.n_levels; ++h) {
            int cnt = 0;
            for (int s = 0; s < ns; ++s) cnt += is_root(s, h);
            if (cnt >= target_tasks) H = h;                       // largest h meeting the target
            if (cnt > best_n || (cnt == best_n && cnt > 0)) { best_n = cnt; best_h = h; }
        }
        if (H == 0) H = best_h;
    }
    P->task_height = H;
    std::vector<char> in_task(ns, 0);
    std::vector<std::pair<double, int>> roots;
    if (H > 0)
        for (int s = 0; s < ns; ++s)
            if (is_root(s, H)) {
                double work = 0.0;
                for (int t = fd[s]; t <= s; ++t) {
                    in_task[t] = 1;
                    work += (double)f[t] * f[t] * S.sn_ncol[t];
                    P->task_max_f = std::max(P->task_max_f, f[t]);
                }
                roots.push_back({work, s});
            }
    // heaviest tasks first (they start in the first wave)
    std::sort(roots.begin(), roots.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (const auto& r : roots) {
        P->task.push_back(fd[r.second]);
        P->task.push_back(r.second);
    }
    // remaining supernodes by level
    P->levels.assign(S.n_levels, LevelPlan());
    std::vector<std::vector<int>> byl(S.n_levels);
    for (int s = 0; s < ns; ++s)
        if (!in_task[s]) byl[lev[s]].push_back(s);
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
        for (int t = 0; t < L.n_warp; t += 4) {
            const int g = (int)P->fwg_ptr.size() - 1;
            P->fwg_ptr.push_back(L.off_warp + std::min(t + 4, L.n_warp));
            P->fitems.push_back((g << 2) | 1);
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
