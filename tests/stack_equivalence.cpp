// The batch analysis assembled from distinct instance patterns (stack_analysis) against
// the analysis of the whole block-diagonal stack with the instances' orderings
// concatenated: every array of the KKT pattern and of the supernodal analysis must be
// equal.  Built by tests/test_stack_equivalence.py from the library's host sources.
//
// Input (binary, int32 unless noted): nb, then per instance n m p l nsoc q[nsoc] and the
// CSC matrices P, A, G, each as rows cols nnz colptr[cols+1] rowidx[nnz] val[nnz] (f64).
// Arguments: <input file> <ordering: 1 AMD, 2 ND> [plant] — with `plant` one assembly
// slot of the assembled analysis is moved first (a control: the comparison must fail).
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "symbolic.h"

using namespace qoco;

namespace {

struct Mat {
    int rows = 0, cols = 0, nnz = 0;
    std::vector<int> p, i;
    std::vector<double> v;
    qoco_csc c{};
};

struct Inst {
    int n, m, p, l, nsoc;
    std::vector<int> q;
    Mat P, A, G;
};

FILE* g_in;
template <class T>
void rd(T* d, size_t n) {
    if (n && fread(d, sizeof(T), n, g_in) != n) {
        std::printf("FAIL short input\n");
        std::exit(2);
    }
}

Mat read_mat() {
    Mat M;
    int h[3];
    rd(h, 3);
    M.rows = h[0]; M.cols = h[1]; M.nnz = h[2];
    M.p.resize(M.cols + 1); rd(M.p.data(), M.p.size());
    M.i.resize(M.nnz); rd(M.i.data(), M.i.size());
    M.v.resize(M.nnz); rd(M.v.data(), M.v.size());
    M.c = qoco_csc{M.rows, M.cols, M.nnz, M.p.data(), M.i.data(), M.v.data()};
    return M;
}

int fails = 0;
template <class A, class B>
void same(const char* what, const A& a, const B& b) {
    bool ok = a.size() == b.size();
    for (size_t k = 0; ok && k < a.size(); ++k) ok = a[k] == b[k];
    if (!ok) {
        ++fails;
        std::printf("FAIL %s (%zu vs %zu entries)\n", what, a.size(), b.size());
    }
}
void same_scalar(const char* what, double a, double b) {
    if (a != b) {
        ++fails;
        std::printf("FAIL %s (%g vs %g)\n", what, a, b);
    }
}

}  // namespace

int main(int argc, char** argv) {
    if (argc < 3) return 2;
    g_in = std::fopen(argv[1], "rb");
    if (!g_in) return 2;
    const int ordering = std::atoi(argv[2]);
    int nb;
    rd(&nb, 1);
    std::vector<Inst> I(nb);
    for (Inst& x : I) {
        int h[5];
        rd(h, 5);
        x.n = h[0]; x.m = h[1]; x.p = h[2]; x.l = h[3]; x.nsoc = h[4];
        x.q.resize(x.nsoc);
        rd(x.q.data(), x.q.size());
        x.P = read_mat(); x.A = read_mat(); x.G = read_mat();
    }
    std::fclose(g_in);

    // the stack: x and y in instance order, every orthant row, then every SOC row
    StackLayout L;
    L.xo = L.yo = L.lo = L.so = L.ko = {0};
    L.Poff = L.Aoff = L.Goff = {0};
    for (const Inst& x : I) { L.n += x.n; L.p += x.p; L.m += x.m; L.l += x.l; }
    for (const Inst& x : I) {
        L.xo.push_back(L.xo.back() + x.n);
        L.yo.push_back(L.yo.back() + x.p);
        L.lo.push_back(L.lo.back() + x.l);
        L.so.push_back(L.so.back() + x.m - x.l);
        L.ko.push_back(L.ko.back() + x.nsoc);
        L.Poff.push_back(L.Poff.back() + x.P.nnz);
        L.Aoff.push_back(L.Aoff.back() + x.A.nnz);
        L.Goff.push_back(L.Goff.back() + x.G.nnz);
    }
    std::vector<int> Pp{0}, Pi, Ap{0}, Ai, Gp{0}, Gi, q;
    std::vector<double> Pv, Av, Gv;
    for (int k = 0; k < nb; ++k) {
        const Inst& x = I[k];
        for (int j = 0; j < x.n; ++j) {
            for (int t = x.P.p[j]; t < x.P.p[j + 1]; ++t) { Pi.push_back(L.xo[k] + x.P.i[t]); Pv.push_back(x.P.v[t]); }
            Pp.push_back((int)Pi.size());
            for (int t = x.A.p[j]; t < x.A.p[j + 1]; ++t) { Ai.push_back(L.yo[k] + x.A.i[t]); Av.push_back(x.A.v[t]); }
            Ap.push_back((int)Ai.size());
            for (int t = x.G.p[j]; t < x.G.p[j + 1]; ++t) {
                const int r = x.G.i[t];
                Gi.push_back(r < x.l ? L.lo[k] + r : L.l + L.so[k] + (r - x.l));
                Gv.push_back(x.G.v[t]);
            }
            Gp.push_back((int)Gi.size());
        }
        q.insert(q.end(), x.q.begin(), x.q.end());
    }
    qoco_csc Ps{L.n, L.n, (int)Pi.size(), Pp.data(), Pi.data(), Pv.data()};
    qoco_csc As{L.p, L.n, (int)Ai.size(), Ap.data(), Ai.data(), Av.data()};
    qoco_csc Gs{L.m, L.n, (int)Gi.size(), Gp.data(), Gi.data(), Gv.data()};
    KKTPattern KS;
    build_kkt_pattern(&KS, L.n, L.m, L.p, Pi.empty() ? nullptr : &Ps, L.p ? &As : nullptr, &Gs, L.l,
                      (int)q.size(), q.data());

    // distinct patterns (equal KKT patterns of equal layouts), ordered and analysed once
    qoco_gpu_settings st{};
    st.ordering = ordering;
    std::vector<KKTPattern> pats;
    std::vector<int> cls(nb), cnt;
    for (int k = 0; k < nb; ++k) {
        const Inst& x = I[k];
        KKTPattern K1;
        build_kkt_pattern(&K1, x.n, x.m, x.p, x.P.nnz ? &x.P.c : nullptr, x.p ? &x.A.c : nullptr, &x.G.c, x.l,
                          x.nsoc, x.q.data());
        int c = -1;
        for (size_t j = 0; j < pats.size() && c < 0; ++j)
            if (pats[j].n == K1.n && pats[j].p == K1.p && pats[j].l == K1.l && pats[j].q == K1.q &&
                pats[j].rowptr == K1.rowptr && pats[j].colidx == K1.colidx && pats[j].src == K1.src)
                c = (int)j;
        if (c < 0) {
            c = (int)pats.size();
            pats.push_back(std::move(K1));
            cnt.push_back(0);
        }
        cls[k] = c;
        ++cnt[c];
    }
    std::vector<std::vector<int>> perms;
    const int used = order_batch_patterns(pats, cnt, st, nb, &perms);
    std::vector<Symbolic> syms(pats.size());
    for (size_t c = 0; c < pats.size(); ++c) analyze(pats[c], st, &syms[c], 1, &perms[c], used);
    KKTPattern K;
    Symbolic S;
    stack_analysis(pats, syms, cls, L, q, Pv.data(), Av.data(), Gv.data(), &K, &S);

    if (argc > 3 && std::string(argv[3]) == "plant" && !S.amap_slot.empty()) S.amap_slot.back() += 1;

    // the reference: the whole stack analysed with the concatenated orderings
    std::vector<int> perm0;
    for (int k = 0; k < nb; ++k)
        for (int o : perms[cls[k]]) perm0.push_back(L.row(k, o));
    Symbolic R;
    analyze(KS, st, &R, nb, &perm0, used);

    same("rowptr", K.rowptr, KS.rowptr);
    same("colidx", K.colidx, KS.colidx);
    same("src", K.src, KS.src);
    same("val0", K.val0, KS.val0);
    same("diag_slot", K.diag_slot, KS.diag_slot);
    same("w2_slot", K.w2_slot, KS.w2_slot);
    same("w2_ptr", K.w2_ptr, KS.w2_ptr);
    same("sign", K.sign, KS.sign);
    same("cone_off", K.cone_off, KS.cone_off);
    same("q", K.q, KS.q);
    same_scalar("N", K.N, KS.N);
    same_scalar("nnzP", (double)K.nnzP, (double)KS.nnzP);
    same_scalar("nnzA", (double)K.nnzA, (double)KS.nnzA);
    same_scalar("nnzG", (double)K.nnzG, (double)KS.nnzG);
    same("perm", S.perm, R.perm);
    same("iperm", S.iperm, R.iperm);
    same_scalar("ns", S.ns, R.ns);
    same("sn_first", S.sn_first, R.sn_first);
    same("sn_ncol", S.sn_ncol, R.sn_ncol);
    same("sn_nrow", S.sn_nrow, R.sn_nrow);
    same("sn_parent", S.sn_parent, R.sn_parent);
    same("row_ptr", S.row_ptr, R.row_ptr);
    same("rows", S.rows, R.rows);
    same("front_off", S.front_off, R.front_off);
    same("upd_off", S.upd_off, R.upd_off);
    same("rel", S.rel, R.rel);
    same("child_ptr", S.child_ptr, R.child_ptr);
    same("child", S.child, R.child);
    same("level", S.level, R.level);
    same_scalar("n_levels", S.n_levels, R.n_levels);
    same("level_ptr", S.level_ptr, R.level_ptr);
    same("level_list", S.level_list, R.level_list);
    same("amap_ptr", S.amap_ptr, R.amap_ptr);
    same("amap_slot", S.amap_slot, R.amap_slot);
    same("amap_off", S.amap_off, R.amap_off);
    same("dsign", S.dsign, R.dsign);
    same_scalar("l_nnz", (double)S.l_nnz, (double)R.l_nnz);
    same_scalar("flops", S.flops, R.flops);
    same_scalar("max_front", S.max_front, R.max_front);
    same_scalar("front_entries", (double)S.front_entries, (double)R.front_entries);
    if (fails) {
        std::printf("%d differences\n", fails);
        return 1;
    }
    std::printf("ok instances=%d patterns=%zu N=%d supernodes=%d\n", nb, pats.size(), K.N, S.ns);
    return 0;
}
