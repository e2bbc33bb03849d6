// Structural checks of the host symbolic analysis (ordering, supernodes, row structures,
// relative indices, assembly map) and of the launch plan (every front in exactly one
// factor list and one solve list; dataflow items in topological order, the condition
// under which their bounded waits always end) that the device kernels rely on.  Built and
// run by tests/test_host_invariants.py on the CPU.
//
// usage: host_invariants <problem dir> <ordering> <trees> [plant_rel | plant_map]
// The problem directory holds dims.bin (n, m, p, l, nsoc, q…) and for P (upper), A, G:
// <M>_hdr.bin (rows, cols, nnz), <M>_p.bin (colptr), <M>_i.bin (rowidx), <M>_x.bin (values).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <string>
#include <vector>

#include "plan.h"
#include "qoco_gpu.h"
#include "symbolic.h"

using namespace qoco;

namespace {

template <class T>
std::vector<T> read_all(const std::string& f) {
    std::ifstream in(f, std::ios::binary | std::ios::ate);
    if (!in) return {};
    const size_t n = (size_t)in.tellg();
    in.seekg(0);
    std::vector<T> v(n / sizeof(T));
    in.read((char*)v.data(), (std::streamsize)n);
    return v;
}

struct Csc {
    std::vector<int> hdr, p, i;
    std::vector<double> x;
    qoco_csc c{};
};

Csc load(const std::string& d, const char* name) {
    Csc m;
    m.hdr = read_all<int>(d + "/" + name + "_hdr.bin");
    m.p = read_all<int>(d + "/" + name + "_p.bin");
    m.i = read_all<int>(d + "/" + name + "_i.bin");
    m.x = read_all<double>(d + "/" + name + "_x.bin");
    m.c = {m.hdr[0], m.hdr[1], m.hdr[2], m.p.data(), m.i.data(), m.x.data()};
    return m;
}

int fails = 0;
void check(bool ok, const char* what, long a = -1, long b = -1) {
    if (ok) return;
    if (fails < 20) std::printf("FAIL %s (%ld, %ld)\n", what, a, b);
    ++fails;
}

}  // namespace

int main(int argc, char** argv) {
    if (argc < 4) return 2;
    const std::string d = argv[1];
    const int ordering = std::atoi(argv[2]), trees = std::atoi(argv[3]);
    const std::vector<int> dims = read_all<int>(d + "/dims.bin");
    Csc P = load(d, "P"), A = load(d, "A"), G = load(d, "G");
    const int n = dims[0], m = dims[1], p = dims[2], l = dims[3], nsoc = dims[4];
    std::string msg;
    if (validate_problem(n, m, p, P.c.nnz ? &P.c : nullptr, nullptr, p ? &A.c : nullptr, nullptr, &G.c,
                         nullptr, l, nsoc, dims.data() + 5, false, &msg)) {
        std::printf("FAIL validation: %s\n", msg.c_str());
        return 1;
    }
    KKTPattern K;
    build_kkt_pattern(&K, n, m, p, P.c.nnz ? &P.c : nullptr, p ? &A.c : nullptr, &G.c, l, nsoc, dims.data() + 5);
    qoco_gpu_settings st{};  // the analysis reads the ordering and the ND leaf size only
    st.ordering = ordering;
    st.nd_leaf = 64;
    Symbolic S;
    analyze(K, st, &S, trees);
    const int N = K.N, ns = S.ns;
    // self-test of the checker: a planted error in one relative index or map offset
    if (argc > 4 && std::string(argv[4]) == "plant_rel" && !S.rel.empty()) S.rel[S.rel.size() / 2] ^= 1;
    if (argc > 4 && std::string(argv[4]) == "plant_map" && !S.amap_off.empty()) S.amap_off[S.amap_off.size() / 2] += 1;

    // KKT pattern: rows sorted, every diagonal present, symmetric
    for (int i = 0; i < N; ++i) {
        for (int64_t t = K.rowptr[i] + 1; t < K.rowptr[i + 1]; ++t)
            check(K.colidx[t - 1] < K.colidx[t], "KKT row sorted", i, (long)t);
        check(K.diag_slot[i] >= 0 && K.colidx[K.diag_slot[i]] == i, "KKT diagonal", i);
    }
    auto slot_of = [&](int i, int j) -> int64_t {
        const int* lo = K.colidx.data() + K.rowptr[i];
        const int* hi = K.colidx.data() + K.rowptr[i + 1];
        const int* it = std::lower_bound(lo, hi, j);
        return (it != hi && *it == j) ? (int64_t)(it - K.colidx.data()) : -1;
    };
    for (int i = 0; i < N; ++i)
        for (int64_t t = K.rowptr[i]; t < K.rowptr[i + 1]; ++t)
            check(slot_of(K.colidx[t], i) >= 0, "KKT symmetric", i, K.colidx[t]);

    // ordering
    std::vector<int> seen(N, 0);
    for (int j = 0; j < N; ++j) {
        check(S.perm[j] >= 0 && S.perm[j] < N && !seen[S.perm[j]]++, "perm is a permutation", j);
        check(S.iperm[S.perm[j]] == j, "iperm inverts perm", j);
        check(S.dsign[j] == K.sign[S.perm[j]], "pivot sign", j);
    }

    // supernodes: contiguous columns, children before parents, consistent child lists
    check(S.sn_first[0] == 0 && S.sn_first[ns] == N, "supernodes cover the columns");
    for (int s = 0; s < ns; ++s) {
        check(S.sn_first[s + 1] > S.sn_first[s], "supernode not empty", s);
        check(S.sn_ncol[s] == S.sn_first[s + 1] - S.sn_first[s], "supernode width", s);
        check(S.sn_parent[s] == -1 || S.sn_parent[s] > s, "postorder", s, S.sn_parent[s]);
    }
    for (int s = 0; s < ns; ++s)
        for (int k = S.child_ptr[s]; k < S.child_ptr[s + 1]; ++k)
            check(S.sn_parent[S.child[k]] == s, "child list", s, S.child[k]);
    {
        std::vector<int> nch(ns, 0);
        for (int s = 0; s < ns; ++s)
            if (S.sn_parent[s] >= 0) nch[S.sn_parent[s]]++;
        for (int s = 0; s < ns; ++s) check(nch[s] == S.child_ptr[s + 1] - S.child_ptr[s], "child count", s);
    }

    // row structures: own columns first, then strictly increasing rows below
    std::vector<int> pos(N, -1);
    for (int s = 0; s < ns; ++s) {
        const int first = S.sn_first[s], c = S.sn_ncol[s], last = first + c - 1;
        const int64_t r0 = S.row_ptr[s], r1 = S.row_ptr[s + 1];
        check(S.sn_nrow[s] == (int)(r1 - r0), "front order", s);
        for (int k = 0; k < c; ++k) check(S.rows[r0 + k] == first + k, "own columns first", s, k);
        for (int64_t t = r0 + c; t < r1; ++t) {
            check(S.rows[t] > last, "update rows below", s, (long)t);
            if (t > r0 + c) check(S.rows[t] > S.rows[t - 1], "update rows sorted", s, (long)t);
        }
        check(S.front_off[s + 1] - S.front_off[s] == (int64_t)S.sn_nrow[s] * S.sn_nrow[s], "front offsets", s);
        check(S.upd_off[s + 1] - S.upd_off[s] == S.sn_nrow[s] - c, "update offsets", s);
    }

    // the structure of L contains the matrix: entry (i, j), i > j, of the permuted KKT lies
    // in the rows of j's supernode
    for (int s = 0; s < ns; ++s) {
        for (int64_t t = S.row_ptr[s]; t < S.row_ptr[s + 1]; ++t) pos[S.rows[t]] = (int)(t - S.row_ptr[s]);
        for (int j = S.sn_first[s]; j < S.sn_first[s + 1]; ++j) {
            const int o = S.perm[j];
            for (int64_t t = K.rowptr[o]; t < K.rowptr[o + 1]; ++t) {
                const int i = S.iperm[K.colidx[t]];
                if (i > j) check(pos[i] >= 0, "matrix entry inside the front", i, j);
            }
        }
        // children's update rows are rows of the parent, at their relative index
        for (int k = S.child_ptr[s]; k < S.child_ptr[s + 1]; ++k) {
            const int ch = S.child[k], cc = S.sn_ncol[ch];
            for (int64_t t = S.row_ptr[ch] + cc; t < S.row_ptr[ch + 1]; ++t) {
                const int64_t u = S.upd_off[ch] + (t - S.row_ptr[ch] - cc);
                check(pos[S.rows[t]] >= 0, "child row in parent", ch, S.rows[t]);
                check(S.rel[u] == pos[S.rows[t]], "relative index", ch, (long)u);
            }
        }
        for (int64_t t = S.row_ptr[s]; t < S.row_ptr[s + 1]; ++t) pos[S.rows[t]] = -1;
    }

    // assembly map: every lower entry of the permuted KKT exactly once, at its front position
    std::vector<int> hits(K.colidx.size(), 0);
    for (int s = 0; s < ns; ++s) {
        const int f = S.sn_nrow[s], c = S.sn_ncol[s], first = S.sn_first[s];
        const int64_t r0 = S.row_ptr[s];
        for (int64_t e = S.amap_ptr[s]; e < S.amap_ptr[s + 1]; ++e) {
            const int64_t off = S.amap_off[e];
            const int col = (int)(off / f), row = (int)(off - (int64_t)col * f);
            const int64_t slot = S.amap_slot[e];
            check(col >= 0 && col < c && row >= col && row < f, "map offset in the front's lower part", s, off);
            if (!(col >= 0 && col < c && row >= col && row < f)) continue;
            const int o = S.perm[first + col];
            check(slot >= K.rowptr[o] && slot < K.rowptr[o + 1], "map slot in the column's KKT row", s, (long)slot);
            check(S.iperm[K.colidx[slot]] == S.rows[r0 + row], "map slot's row", s, (long)slot);
            hits[slot]++;
        }
    }
    for (int i = 0; i < N; ++i)
        for (int64_t t = K.rowptr[i]; t < K.rowptr[i + 1]; ++t) {
            const bool lower = S.iperm[K.colidx[t]] >= S.iperm[i];
            check(hits[t] == (lower ? 1 : 0), "lower entries mapped once", i, (long)t);
        }

    // levels: leaves 0, a parent above each child
    int maxlev = 0;
    for (int s = 0; s < ns; ++s) {
        if (S.child_ptr[s + 1] == S.child_ptr[s]) check(S.level[s] == 0, "leaf level", s);
        if (S.sn_parent[s] >= 0) check(S.level[S.sn_parent[s]] > S.level[s], "parent above child", s);
        maxlev = std::max(maxlev, S.level[s]);
    }
    check(S.n_levels == maxlev + 1, "level count");
    // launch plan
    int df_solve_checked = 0, df_factor_checked = 0;
    int kinds[4] = {0, 0, 0, 0};  // dataflow factorisation items of each kind
    {
        PlanHost P;
        build_plan(S, &P);
        std::vector<int> fcount(ns, 0), scount(ns, 0);
        for (const std::vector<int>* L : {&P.thread, &P.warp, &P.small, &P.large, &P.big})
            for (int x : *L) fcount[x]++;
        for (const std::vector<int>* L : {&P.sthread, &P.swarp, &P.cta, &P.big})
            for (int x : *L) scount[x]++;
        for (int x = 0; x < ns; ++x) {
            check(fcount[x] == 1, "front in one factor list", x, fcount[x]);
            check(scount[x] == 1, "front in one solve list", x, scount[x]);
        }
        for (size_t lv = 0; lv < P.levels.size(); ++lv) {
            const LevelPlan& L = P.levels[lv];
            for (int t = 0; t < L.n_sthread; ++t) check(S.level[P.sthread[L.off_sthread + t]] == (int)lv, "level list", (long)lv);
            for (int t = 0; t < L.n_swarp; ++t) check(S.level[P.swarp[L.off_swarp + t]] == (int)lv, "level list", (long)lv);
        }
        // dataflow solve items: children strictly before parents
        if (P.cta.empty() && P.big.empty()) {
            ++df_solve_checked;
            std::vector<int> item_of(ns, -1);
            for (size_t it = 0; it < P.items.size(); ++it) {
                const int item = P.items[it];
                if (item >= 0) { check(item_of[item] < 0, "solve item once", item); item_of[item] = (int)it; continue; }
                const int b = -item - 1;
                for (int t = P.tb_ptr[b]; t < P.tb_ptr[b + 1]; ++t) {
                    check(item_of[P.sthread[t]] < 0, "solve item once", P.sthread[t]);
                    item_of[P.sthread[t]] = (int)it;
                }
            }
            for (int x = 0; x < ns; ++x) {
                check(item_of[x] >= 0, "solve item covers the front", x);
                if (S.sn_parent[x] >= 0) check(item_of[x] < item_of[S.sn_parent[x]], "solve items topological", x);
            }
        }
        // dataflow factorisation items
        if (P.large.empty() && P.big.empty()) {
            ++df_factor_checked;
            std::vector<int> item_of(ns, -1);
            for (size_t it = 0; it < P.fitems.size(); ++it) {
                const int kind = P.fitems[it] & 3, idx = P.fitems[it] >> 2;
                std::vector<int> members;
                // 0: a batch of one-thread fronts; 1: a group of warp fronts; 3: a group of
                // fronts two to a warp; 2: one CTA front
                if (kind == 0) for (int t = P.ftb_ptr[idx]; t < P.ftb_ptr[idx + 1]; ++t) members.push_back(P.thread[t]);
                else if (kind == 1 || kind == 3) {
                    for (int t = P.fwg_ptr[idx]; t < P.fwg_ptr[idx + 1]; ++t) {
                        members.push_back(P.warp[t]);
                        if (kind == 3) check(P.warp[t] >= 0 && S.sn_nrow[P.warp[t]] <= kPairFront, "pair front order", t);
                    }
                } else members.push_back(idx);
                ++kinds[kind];
                for (int x : members) {
                    check(x >= 0 && x < ns, "factor item front index", x);
                    if (x < 0 || x >= ns) continue;
                    check(item_of[x] < 0, "factor item once", x);
                    item_of[x] = (int)it;
                }
            }
            for (int x = 0; x < ns; ++x) {
                check(item_of[x] >= 0, "factor item covers the front", x);
                if (S.sn_parent[x] >= 0) check(item_of[x] < item_of[S.sn_parent[x]], "factor items topological", x);
            }
        }
    }
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("ok N=%d supernodes=%d levels=%d dataflow plans checked: solve %d factor %d items %d %d %d %d\n",
                N, ns, S.n_levels, df_solve_checked, df_factor_checked, kinds[0], kinds[1], kinds[2], kinds[3]);
    return 0;
}
