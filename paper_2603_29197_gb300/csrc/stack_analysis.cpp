// KKT pattern and supernodal analysis of a batch's block-diagonal stack, assembled from
// the analyses of its distinct instance patterns (set-up phase, host).
//
// A batch of MPC instances holds a few dozen distinct sparsity patterns among thousands
// of instances.  Each pattern's KKT pattern is built, ordered and analysed once; the
// stack's arrays are then written instance by instance, each a relabelled copy of its
// pattern's: rows and columns through the instance's place in the stack, supernodes,
// row structures, front and update offsets, children and assembly slots shifted by the
// instances before it.  The copy is exact: on the stack with the instances' orderings
// concatenated, the elimination forest is postordered tree by tree (an instance's
// columns stay contiguous and in its own order), fundamental supernodes, amalgamation
// and absorption never merge across trees, and the map from local to stack rows is
// increasing, so every sorted row of K stays sorted and keeps its slots' order.
#include <algorithm>
#include <thread>

#include "symbolic.h"

namespace qoco {

namespace {

// f(i0, i1) over contiguous instance ranges on a few host threads; the callers write
// disjoint parts of preallocated arrays, so the result does not depend on the split
template <class F>
void over_instances(int nb, F f) {
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nth = std::max(1, std::min({16, hw, nb / 64 + 1}));
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t)
        pool.emplace_back([&, t]() { f((int)((int64_t)nb * t / nth), (int)((int64_t)nb * (t + 1) / nth)); });
    f(0, (int)((int64_t)nb / nth));
    for (auto& th : pool) th.join();
}

}  // namespace

void stack_analysis(const std::vector<KKTPattern>& pats, const std::vector<Symbolic>& syms,
                    const std::vector<int>& cls, const StackLayout& L, const std::vector<int>& q,
                    const double* Pv, const double* Av, const double* Gv, KKTPattern* K, Symbolic* S) {
    const int nb = L.nb();
    const int n = L.n, p = L.p, m = L.m, N = n + p + m;
    const int nsoc = (int)q.size();

    // ---- the KKT pattern ----------------------------------------------------------
    K->n = n; K->m = m; K->p = p; K->l = L.l; K->nsoc = nsoc; K->N = N;
    K->q = q;
    K->cone_off.resize(nsoc);
    for (int k = 0, o = L.l; k < nsoc; ++k) { K->cone_off[k] = o; o += q[k]; }
    K->nnzP = L.Poff[nb];
    K->nnzA = L.Aoff[nb];
    K->nnzG = L.Goff[nb];
    K->rowptr.assign((size_t)N + 1, 0);
    over_instances(nb, [&](int i0, int i1) {
        for (int i = i0; i < i1; ++i) {
            const KKTPattern& P = pats[cls[i]];
            for (int r = 0; r < P.N; ++r) K->rowptr[L.row(i, r) + 1] = P.rowptr[r + 1] - P.rowptr[r];
        }
    });
    for (int g = 0; g < N; ++g) K->rowptr[g + 1] += K->rowptr[g];
    const int64_t nnz = K->rowptr[N];
    K->colidx.resize(nnz);
    K->src.resize(nnz);
    K->val0.resize(nnz);
    K->diag_slot.resize(N);
    K->sign.resize(N);
    const int64_t oA = K->nnzP, oG = K->nnzP + K->nnzA;
    over_instances(nb, [&](int i0, int i1) {
        for (int i = i0; i < i1; ++i) {
            const KKTPattern& P = pats[cls[i]];
            const int64_t pA = P.nnzP, pG = P.nnzP + P.nnzA;
            for (int r = 0; r < P.N; ++r) {
                const int g = L.row(i, r);
                int64_t at = K->rowptr[g];
                for (int64_t t = P.rowptr[r]; t < P.rowptr[r + 1]; ++t, ++at) {
                    K->colidx[at] = L.row(i, P.colidx[t]);
                    // the instance's data index → the stack's [P | A | G] value index
                    const int64_t s = P.src[t];
                    int64_t gs = -1;
                    double v = 0.0;
                    if (s >= 0 && s < pA) { gs = L.Poff[i] + s; v = Pv[gs]; }
                    else if (s >= pA && s < pG) { gs = oA + L.Aoff[i] + (s - pA); v = Av[gs - oA]; }
                    else if (s >= pG) { gs = oG + L.Goff[i] + (s - pG); v = Gv[gs - oG]; }
                    K->src[at] = gs;
                    K->val0[at] = v;
                }
                K->diag_slot[g] = K->rowptr[g] + (P.diag_slot[r] - P.rowptr[r]);
                K->sign[g] = g < n ? 1 : -1;
            }
        }
    });
    // −W² slots: the orthant diagonals in the stack's orthant order, then each SOC's
    // dense block (row-major) in the stack's SOC order
    K->w2_ptr.assign((size_t)nsoc + 1, 0);
    for (int k = 0; k < nsoc; ++k) K->w2_ptr[k + 1] = K->w2_ptr[k] + (int64_t)q[k] * q[k];
    K->w2_slot.resize((size_t)L.l + K->w2_ptr[nsoc]);
    over_instances(nb, [&](int i0, int i1) {
        for (int i = i0; i < i1; ++i) {
            const KKTPattern& P = pats[cls[i]];
            const int li = L.lo[i + 1] - L.lo[i];
            for (int r = 0; r < li; ++r) K->w2_slot[L.lo[i] + r] = K->diag_slot[n + p + L.lo[i] + r];
            for (int k = 0; k < P.nsoc; ++k) {
                const int qk = P.q[k];
                const int64_t dst = L.l + K->w2_ptr[L.ko[i] + k];
                for (int e = 0; e < qk * qk; ++e) {
                    const int r = P.n + P.p + P.cone_off[k] + e / qk;
                    const int64_t t = P.w2_slot[P.l + P.w2_ptr[k] + e];
                    K->w2_slot[dst + e] = K->rowptr[L.row(i, r)] + (t - P.rowptr[r]);
                }
            }
        }
    });

    // ---- the supernodal analysis ---------------------------------------------------
    // per-instance offsets of columns, supernodes and every per-supernode array
    std::vector<int> col_o(nb + 1, 0), sn_o(nb + 1, 0);
    std::vector<int64_t> row_o(nb + 1, 0), front_o(nb + 1, 0), upd_o(nb + 1, 0), child_o(nb + 1, 0),
        amap_o(nb + 1, 0);
    S->l_nnz = 0;
    S->flops = 0.0;
    S->max_front = 0;
    S->n_levels = 0;
    for (int i = 0; i < nb; ++i) {
        const Symbolic& Y = syms[cls[i]];
        col_o[i + 1] = col_o[i] + Y.N;
        sn_o[i + 1] = sn_o[i] + Y.ns;
        row_o[i + 1] = row_o[i] + Y.row_ptr[Y.ns];
        front_o[i + 1] = front_o[i] + Y.front_off[Y.ns];
        upd_o[i + 1] = upd_o[i] + Y.upd_off[Y.ns];
        child_o[i + 1] = child_o[i] + Y.child_ptr[Y.ns];
        amap_o[i + 1] = amap_o[i] + Y.amap_ptr[Y.ns];
        S->l_nnz += Y.l_nnz;
        S->flops += Y.flops;
        S->max_front = std::max(S->max_front, Y.max_front);
        S->n_levels = std::max(S->n_levels, Y.n_levels);
    }
    const int ns = sn_o[nb];
    S->N = N;
    S->ns = ns;
    S->perm.resize(N);
    S->iperm.resize(N);
    S->dsign.resize(N);
    S->sn_first.resize((size_t)ns + 1);
    S->sn_ncol.resize(ns);
    S->sn_nrow.resize(ns);
    S->sn_parent.resize(ns);
    S->level.resize(ns);
    S->row_ptr.resize((size_t)ns + 1);
    S->rows.resize(row_o[nb]);
    S->front_off.resize((size_t)ns + 1);
    S->upd_off.resize((size_t)ns + 1);
    S->rel.resize(upd_o[nb]);
    S->child_ptr.resize((size_t)ns + 1);
    S->child.resize(child_o[nb]);
    S->amap_ptr.resize((size_t)ns + 1);
    S->amap_slot.resize(amap_o[nb]);
    S->amap_off.resize(amap_o[nb]);
    // each pattern's KKT row of every slot (for the assembly slots)
    std::vector<std::vector<int>> slot_row(pats.size());
    for (size_t c = 0; c < pats.size(); ++c) {
        slot_row[c].resize(pats[c].nnz());
        for (int r = 0; r < pats[c].N; ++r)
            for (int64_t t = pats[c].rowptr[r]; t < pats[c].rowptr[r + 1]; ++t) slot_row[c][t] = r;
    }
    over_instances(nb, [&](int i0, int i1) {
        for (int i = i0; i < i1; ++i) {
            const int c = cls[i];
            const Symbolic& Y = syms[c];
            const KKTPattern& P = pats[c];
            const int co = col_o[i], so = sn_o[i];
            for (int j = 0; j < Y.N; ++j) {
                S->perm[co + j] = L.row(i, Y.perm[j]);
                S->dsign[co + j] = Y.dsign[j];
            }
            for (int s = 0; s < Y.ns; ++s) {
                S->sn_first[so + s] = Y.sn_first[s] + co;
                S->sn_ncol[so + s] = Y.sn_ncol[s];
                S->sn_nrow[so + s] = Y.sn_nrow[s];
                S->sn_parent[so + s] = Y.sn_parent[s] >= 0 ? Y.sn_parent[s] + so : -1;
                S->level[so + s] = Y.level[s];
                S->row_ptr[so + s] = Y.row_ptr[s] + row_o[i];
                S->front_off[so + s] = Y.front_off[s] + front_o[i];
                S->upd_off[so + s] = Y.upd_off[s] + upd_o[i];
                S->child_ptr[so + s] = Y.child_ptr[s] + child_o[i];
                S->amap_ptr[so + s] = Y.amap_ptr[s] + amap_o[i];
            }
            for (int64_t t = 0; t < Y.row_ptr[Y.ns]; ++t) S->rows[row_o[i] + t] = Y.rows[t] + co;
            std::copy(Y.rel.begin(), Y.rel.end(), S->rel.begin() + upd_o[i]);
            for (int64_t t = 0; t < Y.child_ptr[Y.ns]; ++t) S->child[child_o[i] + t] = Y.child[t] + so;
            for (int64_t t = 0; t < Y.amap_ptr[Y.ns]; ++t) {
                const int64_t loc = Y.amap_slot[t];
                const int r = slot_row[c][loc];
                S->amap_slot[amap_o[i] + t] = K->rowptr[L.row(i, r)] + (loc - P.rowptr[r]);
            }
            std::copy(Y.amap_off.begin(), Y.amap_off.end(), S->amap_off.begin() + amap_o[i]);
        }
    });
    S->sn_first[ns] = N;
    S->row_ptr[ns] = row_o[nb];
    S->front_off[ns] = front_o[nb];
    S->upd_off[ns] = upd_o[nb];
    S->child_ptr[ns] = child_o[nb];
    S->amap_ptr[ns] = amap_o[nb];
    S->front_entries = front_o[nb];
    over_instances(nb, [&](int i0, int i1) {
        for (int j = col_o[i0]; j < col_o[i1]; ++j) S->iperm[S->perm[j]] = j;
    });
    // supernodes grouped by level, in supernode order within a level
    S->level_ptr.assign((size_t)S->n_levels + 1, 0);
    for (int s = 0; s < ns; ++s) S->level_ptr[S->level[s] + 1]++;
    for (int k = 0; k < S->n_levels; ++k) S->level_ptr[k + 1] += S->level_ptr[k];
    S->level_list.assign(ns, 0);
    std::vector<int> fill(S->level_ptr.begin(), S->level_ptr.end() - 1);
    for (int s = 0; s < ns; ++s) S->level_list[fill[S->level[s]]++] = s;
    if (ns == 0) S->amap_ptr.assign(1, 0);
}

}  // namespace qoco
