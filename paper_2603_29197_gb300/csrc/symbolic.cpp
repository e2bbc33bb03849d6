// Symbolic supernodal analysis of the permuted KKT matrix (set-up phase).
//
// Steps, all on the host, once per sparsity pattern:
//   1. elimination tree of the permuted matrix (Liu's ancestor algorithm with path
//      compression) and a postorder, composed into the ordering;
//   2. column counts of L by row-subtree marking (each row i walks from every k with
//      K_ik ≠ 0, k < i, up the tree until an already-marked node);
//   3. fundamental supernodes (j+1 continues j's supernode when it is j's parent,
//      has j as only child and count(j) = count(j+1) + 1), then relaxed
//      amalgamation of a supernode with its last child when few explicit zeros
//      are added, then absorption of thin children with large updates into their
//      (large) parents, with the columns re-emitted in a topological order;
//   4. row structures R_s (own columns, then the rows below), the supernodal tree,
//      levels (height above the leaves), front/update offsets, the extend-add
//      relative indices and the map from KKT value slots to front positions.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>

#include "symbolic.h"

namespace qoco {

namespace {

std::vector<int> etree(const Graph& g, const std::vector<int>& perm, const std::vector<int>& iperm) {
    const int N = g.N;
    std::vector<int> parent(N, -1), anc(N, -1);
    for (int j = 0; j < N; ++j) {
        int o = perm[j];
        for (int64_t t = g.ptr[o]; t < g.ptr[o + 1]; ++t) {
            int i = iperm[g.adj[t]];
            if (i >= j) continue;
            int r = i;
            while (anc[r] != -1 && anc[r] != j) {
                int nx = anc[r];
                anc[r] = j;
                r = nx;
            }
            if (anc[r] == -1) { anc[r] = j; parent[r] = j; }
        }
    }
    return parent;
}

std::vector<int> postorder(const std::vector<int>& parent) {
    const int N = (int)parent.size();
    std::vector<int> head(N, -1), next(N, -1), post;
    post.reserve(N);
    for (int j = N - 1; j >= 0; --j)
        if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = j; }
    std::vector<int> stack;
    for (int r = 0; r < N; ++r) {
        if (parent[r] != -1) continue;
        stack.push_back(r);
        while (!stack.empty()) {
            int v = stack.back();
            int c = head[v];
            if (c == -1) { post.push_back(v); stack.pop_back(); }
            else { head[v] = next[c]; stack.push_back(c); }
        }
    }
    return post;  // post[k] = old index of the k-th node in postorder
}

// below-diagonal counts of every column of L
std::vector<int> col_counts(const Graph& g, const std::vector<int>& perm,
                            const std::vector<int>& iperm, const std::vector<int>& parent) {
    const int N = g.N;
    std::vector<int> cc(N, 0), mark(N, -1);
    for (int i = 0; i < N; ++i) {
        int o = perm[i];
        mark[i] = i;
        for (int64_t t = g.ptr[o]; t < g.ptr[o + 1]; ++t) {
            int k = iperm[g.adj[t]];
            if (k >= i) continue;
            while (mark[k] != i) {
                mark[k] = i;
                cc[k]++;
                k = parent[k];
            }
        }
    }
    return cc;
}

int sn_height_fundamental(const std::vector<int>& parent, const std::vector<int>& cc) {
    // height of the fundamental-supernode tree: a column that continues its only
    // child's supernode adds no level
    const int N = (int)parent.size();
    std::vector<int> nchild(N, 0);
    for (int j = 0; j < N; ++j) if (parent[j] >= 0) nchild[parent[j]]++;
    std::vector<int> h(N, 0);
    int best = 0;
    for (int j = 0; j < N; ++j) {
        int p = parent[j];
        if (p < 0) { best = std::max(best, h[j]); continue; }
        bool cont = p == j + 1 && nchild[p] == 1 && cc[j] == cc[p] + 1;
        h[p] = std::max(h[p], h[j] + (cont ? 0 : 1));
    }
    return best + 1;
}

}  // namespace

namespace {

// An ordering made ready for the supernodal pass: its elimination tree postordered
// (perm, iperm), that tree (parent) and L's column counts (cc), with the cost figures.
struct Evaluated {
    std::vector<int> perm, iperm, parent, cc;
    OrderingCost cost;
};

void evaluate(const Graph& g, const std::vector<int>& perm0, bool keep_identity, Evaluated* E) {
    const int N = g.N;
    std::vector<int> ip0(N);
    for (int j = 0; j < N; ++j) ip0[perm0[j]] = j;
    // tree and counts of perm0; a postorder of that tree is a topological order of it, so
    // the permuted matrix has the same tree and counts, relabelled (Liu 1990)
    std::vector<int> parent0 = etree(g, perm0, ip0);
    std::vector<int> cc0 = col_counts(g, perm0, ip0, parent0);
    std::vector<int> post;
    if (keep_identity) {
        // NATURAL keeps the identity: any order in which every column precedes its etree
        // parent is valid for the supernodal pass
        post.resize(N);
        std::iota(post.begin(), post.end(), 0);
    } else {
        post = postorder(parent0);
    }
    std::vector<int> ipost(N);
    for (int k = 0; k < N; ++k) ipost[post[k]] = k;
    E->perm.resize(N);
    E->iperm.resize(N);
    E->parent.resize(N);
    E->cc.resize(N);
    for (int k = 0; k < N; ++k) {
        E->perm[k] = perm0[post[k]];
        const int p0 = parent0[post[k]];
        E->parent[k] = p0 >= 0 ? ipost[p0] : -1;
        E->cc[k] = cc0[post[k]];
    }
    for (int j = 0; j < N; ++j) E->iperm[E->perm[j]] = j;
    E->cost = OrderingCost();
    for (int j = 0; j < N; ++j) {
        E->cost.l_nnz += E->cc[j];
        E->cost.flops += (double)E->cc[j] * E->cc[j] + 2.0 * E->cc[j];
    }
    E->cost.height = sn_height_fundamental(E->parent, E->cc);
}

}  // namespace

OrderingCost ordering_cost(const KKTPattern& K, const std::vector<int>& perm0) {
    Evaluated E;
    evaluate(kkt_graph(K), perm0, false, &E);
    return E.cost;
}

int nd_leaf_size(const qoco_gpu_settings& st, int N) {
    // automatic: about 1/2048 of the graph, between 64 and 256 nodes.  On a large stage
    // chain AMD orders a leaf of a few stages with less fill than more dissection levels
    // would (trajectory N = 20000, 540k nodes: leaves of 256 take 27 % fewer flops than 64
    // at the same 16-level tree, 65.7 against 67.7 ms to the 1e-7 gap), while a small
    // graph (an MPC instance of ≤ 1260 nodes) keeps leaves of 64 and its short tree
    // (8 levels; 256 would give 11 and a 6 % slower batch)
    if (st.nd_leaf > 0) return st.nd_leaf;
    return std::min(256, std::max(64, N / 2048));
}

bool auto_picks_nd(const OrderingCost& amd, const OrderingCost& nd, const qoco_gpu_settings& st, int trees) {
    // AUTO: cost model = factor flops at an effective FP64 rate plus a per-level latency
    // for the level-scheduled factor and solves.  The independent trees of a batch on the
    // shared kernels overlap their level chains (up to 64 of them are counted), which
    // favours the lower flop counts of AMD there; a batch on the persistent kernel
    // (batch_schedule 0 or 6–12) walks each instance's tree inside one CTA, so an instance's
    // chain of levels counts in full (MPC batch of 4096 on that kernel: ND 63k solves/s
    // against AMD's 59–68k in FP64, 50k against 33k with FP32 fronts).
    const bool persistent = trees > 1 && (st.batch_schedule == 0 || (st.batch_schedule >= 6 && st.batch_schedule <= 12));
    const double overlap = persistent ? 1.0 : (double)std::max(1, std::min(trees, 64));
    auto cost = [&](const OrderingCost& c) { return c.flops / 2e11 + c.height * 4e-5 / overlap; };
    return cost(nd) < cost(amd);
}

int order_batch_patterns(const std::vector<KKTPattern>& pats, const std::vector<int>& count,
                         const qoco_gpu_settings& st, int trees, std::vector<std::vector<int>>* perms) {
    const int np = (int)pats.size();
    const bool both = st.ordering != QOCO_GPU_ORDER_AMD && st.ordering != QOCO_GPU_ORDER_ND;
    std::vector<std::vector<int>> pa(np), pn(np);
    std::vector<OrderingCost> ca(np), cn(np);
    // one pattern per task, on a few host threads (each result depends on its pattern only)
    const int nth = std::max(1, std::min(np, (int)std::min(16u, std::max(1u, std::thread::hardware_concurrency()))));
    auto work = [&](int t0) {
        for (int c = t0; c < np; c += nth) {
            const Graph g = kkt_graph(pats[c]);
            if (st.ordering != QOCO_GPU_ORDER_ND) {
                pa[c] = order_amd(g);
                if (both) ca[c] = ordering_cost(pats[c], pa[c]);
            }
            if (st.ordering != QOCO_GPU_ORDER_AMD) {
                pn[c] = order_nd(g, nd_leaf_size(st, g.N));
                if (both) cn[c] = ordering_cost(pats[c], pn[c]);
            }
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto& t : pool) t.join();
    int used = st.ordering;
    if (both) {
        // the batch's cost: flops add over the instances, the height is the tallest tree's
        OrderingCost A, D;
        for (int c = 0; c < np; ++c) {
            A.flops += count[c] * ca[c].flops;
            D.flops += count[c] * cn[c].flops;
            A.height = std::max(A.height, ca[c].height);
            D.height = std::max(D.height, cn[c].height);
        }
        used = auto_picks_nd(A, D, st, trees) ? QOCO_GPU_ORDER_ND : QOCO_GPU_ORDER_AMD;
    }
    *perms = used == QOCO_GPU_ORDER_ND ? std::move(pn) : std::move(pa);
    return used;
}

int analyze(const KKTPattern& K, const qoco_gpu_settings& st, Symbolic* S, int trees,
            const std::vector<int>* perm0, int perm0_ordering) {
    const int N = K.N;
    Graph g = kkt_graph(K);
    int used = st.ordering;
    Evaluated E;
    if (perm0) {
        evaluate(g, *perm0, false, &E);
        used = perm0_ordering;
    } else if (st.ordering == QOCO_GPU_ORDER_NATURAL) {
        std::vector<int> perm0(N);
        std::iota(perm0.begin(), perm0.end(), 0);
        evaluate(g, perm0, true, &E);
    } else if (st.ordering == QOCO_GPU_ORDER_AMD) {
        evaluate(g, order_amd(g), false, &E);
    } else if (st.ordering == QOCO_GPU_ORDER_ND) {
        evaluate(g, order_nd(g, nd_leaf_size(st, N)), false, &E);
    } else {
        // AUTO: the two candidates are independent, ordered and evaluated on two host
        // threads, and the cheaper by auto_picks_nd's model is kept
        Evaluated En;
        std::thread tn([&]() { evaluate(g, order_nd(g, nd_leaf_size(st, N)), false, &En); });
        evaluate(g, order_amd(g), false, &E);
        tn.join();
        if (auto_picks_nd(E.cost, En.cost, st, trees)) { E = std::move(En); used = QOCO_GPU_ORDER_ND; }
        else used = QOCO_GPU_ORDER_AMD;
    }

    // 1–2. postordered elimination tree and column counts of the chosen ordering
    S->N = N;
    S->perm = std::move(E.perm);
    S->iperm = std::move(E.iperm);
    const std::vector<int>& perm = S->perm;
    const std::vector<int>& ip = S->iperm;
    std::vector<int> parent = std::move(E.parent);
    std::vector<int> cc = std::move(E.cc);
    S->l_nnz = 0;
    S->flops = 0.0;
    for (int j = 0; j < N; ++j) {
        S->l_nnz += cc[j];
        S->flops += (double)cc[j] * cc[j] + 2.0 * cc[j];
    }

    // 3. fundamental supernodes
    std::vector<int> nchild(N, 0);
    for (int j = 0; j < N; ++j) if (parent[j] >= 0) nchild[parent[j]]++;
    std::vector<int> fs_first;
    for (int j = 0; j < N; ++j) {
        bool cont = j > 0 && parent[j - 1] == j && nchild[j] == 1 && cc[j - 1] == cc[j] + 1;
        if (!cont) fs_first.push_back(j);
    }
    const int nf = (int)fs_first.size();
    fs_first.push_back(N);
    std::vector<int> col2f(N);
    for (int s = 0; s < nf; ++s)
        for (int j = fs_first[s]; j < fs_first[s + 1]; ++j) col2f[j] = s;
    std::vector<int> fparent(nf, -1);
    for (int s = 0; s < nf; ++s) {
        int last = fs_first[s + 1] - 1;
        if (parent[last] >= 0) fparent[s] = col2f[parent[last]];
    }
    // relaxed amalgamation: merge the immediately preceding supernode (the last child)
    constexpr int kAmalgSmallFront = 48, kAmalgSmallCap = 40;
    struct SN { int first, ncol, f; double truenz; int fparent; };
    std::vector<SN> stack;
    stack.reserve(nf);
    for (int s = 0; s < nf; ++s) {
        SN cur;
        cur.first = fs_first[s];
        cur.ncol = fs_first[s + 1] - fs_first[s];
        cur.f = cc[cur.first] + 1;
        cur.truenz = 0;
        for (int j = cur.first; j < cur.first + cur.ncol; ++j) cur.truenz += cc[j] + 1;
        cur.fparent = fparent[s];
        while (!stack.empty()) {
            SN& c = stack.back();
            if (c.fparent != s) break;
            int ncol = c.ncol + cur.ncol;
            int f = c.ncol + cur.f;
            double dense = (double)ncol * f - 0.5 * (double)ncol * (ncol - 1);
            double tnz = c.truenz + cur.truenz;
            double zf = 1.0 - tnz / dense;
            // Merging trades explicit zeros (FP64 work) for fewer supernodes and a shallower
            // tree (a shorter dependent chain of fronts).  A parent that is still a small
            // front stays at order ≤ kAmalgSmallCap, so that it remains on the one-warp /
            // one-thread kernels and their occupancy; larger fronts merge by zeros alone.
            bool ok = (ncol <= 4) || (ncol <= 16 && zf <= 0.8) || (ncol <= 48 && zf <= 0.7) || (zf <= 0.3);
            if (cur.f <= kAmalgSmallFront && f > kAmalgSmallCap) ok = false;
            if (!ok) break;
            cur.first = c.first;
            cur.ncol = ncol;
            cur.f = f;
            cur.truenz = tnz;
            stack.pop_back();
        }
        stack.push_back(cur);
    }
    // 3b. absorption into large fronts.  In a dense part of the factor (the lasso's
    // Schur complement on the equality rows) a large front often has children that are
    // thin (a few columns) but whose update blocks are themselves large dense matrices:
    // only the last child is adjacent to the parent, so the pass above leaves the others
    // as separate fronts, each storing an f×f block (mostly its update) and extend-adding
    // it.  A child with at most kAbsorbCols columns and an update of at least
    // kAbsorbRows rows is merged into its parent, as long as the columns merged into a
    // front stay within max(kAbsorbCols, its own columns / 20) (each merged column costs
    // a rank-1 update of the whole merged front).  The merged fronts' columns are then
    // made contiguous by re-emitting the columns in a topological order of the merged
    // tree (external children first, then every member's columns, children before
    // parents).  The natural ordering is kept as given (no re-emission).
    if (used != QOCO_GPU_ORDER_NATURAL) {
        constexpr int kAbsorbRows = 1024, kAbsorbCols = 256;
        const int nsn = (int)stack.size();
        std::vector<int> scol(N);
        for (int t = 0; t < nsn; ++t)
            for (int j = stack[t].first; j < stack[t].first + stack[t].ncol; ++j) scol[j] = t;
        std::vector<int> sp(nsn, -1);
        for (int t = 0; t < nsn; ++t) {
            const int last = stack[t].first + stack[t].ncol - 1;
            if (parent[last] >= 0) sp[t] = scol[parent[last]];
        }
        std::vector<std::vector<int>> kids(nsn);
        for (int t = 0; t < nsn; ++t)
            if (sp[t] >= 0 && stack[t].f - stack[t].ncol >= kAbsorbRows) kids[sp[t]].push_back(t);
        std::vector<int> into(nsn, -1);
        // group totals (members' columns, front order, true entries), built bottom-up
        std::vector<int> gc(nsn), gf(nsn);
        std::vector<double> gt(nsn);
        for (int t = 0; t < nsn; ++t) { gc[t] = stack[t].ncol; gf[t] = stack[t].f; gt[t] = stack[t].truenz; }
        bool any = false;
        for (int t = 0; t < nsn; ++t) {
            if (kids[t].empty()) continue;
            std::vector<int>& k = kids[t];
            std::stable_sort(k.begin(), k.end(), [&](int a, int b) { return gf[a] - gc[a] > gf[b] - gc[b]; });
            const int cap = std::max(kAbsorbCols, stack[t].ncol / 20);
            int took = 0;
            for (int c : k) {
                if (gc[c] > kAbsorbCols || took + gc[c] > cap) continue;
                into[c] = t;
                took += gc[c];
                gc[t] += gc[c];
                gf[t] += gc[c];
                gt[t] += gt[c];
                any = true;
            }
        }
        if (any) {
            // group root of every supernode (a parent comes after its children)
            std::vector<int> root(nsn);
            for (int t = nsn - 1; t >= 0; --t) root[t] = into[t] >= 0 ? root[into[t]] : t;
            std::vector<std::vector<int>> members(nsn), gkids(nsn);
            for (int t = 0; t < nsn; ++t) {
                members[root[t]].push_back(t);
                if (into[t] < 0 && sp[t] >= 0) gkids[root[sp[t]]].push_back(t);
            }
            std::vector<int> order;  // old column indices in the new order
            order.reserve(N);
            std::vector<SN> merged;
            std::vector<std::pair<int, size_t>> st;  // (group, next child)
            for (int t = 0; t < nsn; ++t) {
                if (into[t] >= 0 || sp[t] >= 0) continue;
                st.push_back({t, 0});
                while (!st.empty()) {
                    auto& top = st.back();
                    if (top.second < gkids[top.first].size()) {
                        const int ch = gkids[top.first][top.second++];
                        st.push_back({ch, 0});
                        continue;
                    }
                    const int g2 = top.first;
                    st.pop_back();
                    SN sn2 = stack[g2];
                    sn2.first = (int)order.size();
                    sn2.ncol = gc[g2];
                    sn2.f = gf[g2];
                    sn2.truenz = gt[g2];
                    for (int mbr : members[g2])
                        for (int j = stack[mbr].first; j < stack[mbr].first + stack[mbr].ncol; ++j) order.push_back(j);
                    merged.push_back(sn2);
                }
            }
            std::vector<int> newpos(N);
            for (int k = 0; k < N; ++k) newpos[order[k]] = k;
            std::vector<int> p2(N), c2(N), pm(N);
            for (int j = 0; j < N; ++j) {
                p2[newpos[j]] = parent[j] >= 0 ? newpos[parent[j]] : -1;
                c2[newpos[j]] = cc[j];
            }
            for (int k = 0; k < N; ++k) pm[k] = S->perm[order[k]];
            parent.swap(p2);
            cc.swap(c2);
            S->perm.swap(pm);
            for (int j = 0; j < N; ++j) S->iperm[S->perm[j]] = j;
            stack.swap(merged);
        }
    }
    const int ns = (int)stack.size();
    S->ns = ns;
    S->sn_first.resize(ns + 1);
    S->sn_ncol.resize(ns);
    for (int s = 0; s < ns; ++s) { S->sn_first[s] = stack[s].first; S->sn_ncol[s] = stack[s].ncol; }
    S->sn_first[ns] = N;
    std::vector<int> col2s(N);
    for (int s = 0; s < ns; ++s)
        for (int j = S->sn_first[s]; j < S->sn_first[s + 1]; ++j) col2s[j] = s;
    S->sn_parent.assign(ns, -1);
    for (int s = 0; s < ns; ++s) {
        int last = S->sn_first[s + 1] - 1;
        if (parent[last] >= 0) S->sn_parent[s] = col2s[parent[last]];
    }
    // children lists
    S->child_ptr.assign(ns + 1, 0);
    for (int s = 0; s < ns; ++s) if (S->sn_parent[s] >= 0) S->child_ptr[S->sn_parent[s] + 1]++;
    for (int s = 0; s < ns; ++s) S->child_ptr[s + 1] += S->child_ptr[s];
    S->child.assign(S->child_ptr[ns], 0);
    {
        std::vector<int> fill(S->child_ptr.begin(), S->child_ptr.end() - 1);
        for (int s = 0; s < ns; ++s) if (S->sn_parent[s] >= 0) S->child[fill[S->sn_parent[s]]++] = s;
    }

    // 4. row structures (children before parents: supernodes are in postorder)
    S->row_ptr.assign(ns + 1, 0);
    S->rows.clear();
    S->sn_nrow.resize(ns);
    std::vector<int> mark(N, -1), buf;
    for (int s = 0; s < ns; ++s) {
        int first = S->sn_first[s], last = S->sn_first[s + 1] - 1;
        buf.clear();
        for (int j = first; j <= last; ++j) { buf.push_back(j); mark[j] = s; }
        for (int j = first; j <= last; ++j) {
            int o = perm[j];
            for (int64_t t = g.ptr[o]; t < g.ptr[o + 1]; ++t) {
                int i = ip[g.adj[t]];
                if (i > last && mark[i] != s) { mark[i] = s; buf.push_back(i); }
            }
        }
        for (int k = S->child_ptr[s]; k < S->child_ptr[s + 1]; ++k) {
            int c = S->child[k];
            for (int64_t t = S->row_ptr[c] + S->sn_ncol[c]; t < S->row_ptr[c + 1]; ++t) {
                int i = S->rows[t];
                if (i > last && mark[i] != s) { mark[i] = s; buf.push_back(i); }
            }
        }
        std::sort(buf.begin() + (last - first + 1), buf.end());
        S->rows.insert(S->rows.end(), buf.begin(), buf.end());
        S->row_ptr[s + 1] = (int64_t)S->rows.size();
        S->sn_nrow[s] = (int)buf.size();
    }
    // levels, offsets
    S->level.assign(ns, 0);
    for (int s = 0; s < ns; ++s)
        if (S->sn_parent[s] >= 0)
            S->level[S->sn_parent[s]] = std::max(S->level[S->sn_parent[s]], S->level[s] + 1);
    S->n_levels = 0;
    for (int s = 0; s < ns; ++s) S->n_levels = std::max(S->n_levels, S->level[s] + 1);
    S->level_ptr.assign(S->n_levels + 1, 0);
    for (int s = 0; s < ns; ++s) S->level_ptr[S->level[s] + 1]++;
    for (int k = 0; k < S->n_levels; ++k) S->level_ptr[k + 1] += S->level_ptr[k];
    S->level_list.assign(ns, 0);
    {
        std::vector<int> fill(S->level_ptr.begin(), S->level_ptr.end() - 1);
        for (int s = 0; s < ns; ++s) S->level_list[fill[S->level[s]]++] = s;
    }
    S->front_off.assign(ns + 1, 0);
    S->upd_off.assign(ns + 1, 0);
    S->max_front = 0;
    for (int s = 0; s < ns; ++s) {
        int64_t f = S->sn_nrow[s];
        S->front_off[s + 1] = S->front_off[s] + f * f;
        S->upd_off[s + 1] = S->upd_off[s] + (f - S->sn_ncol[s]);
        S->max_front = std::max(S->max_front, (int)f);
    }
    S->front_entries = S->front_off[ns];
    // relative indices of each child's update rows inside its parent
    S->rel.assign(S->upd_off[ns], 0);
    S->amap_ptr.assign(ns + 1, 0);
    S->amap_slot.clear();
    S->amap_off.clear();
    S->amap_slot.reserve((size_t)(K.nnz() + N) / 2);  // the lower triangle with the diagonal
    S->amap_off.reserve((size_t)(K.nnz() + N) / 2);
    std::vector<int> pos(N, -1);
    for (int s = 0; s < ns; ++s) {
        for (int64_t t = S->row_ptr[s]; t < S->row_ptr[s + 1]; ++t) pos[S->rows[t]] = (int)(t - S->row_ptr[s]);
        for (int k = S->child_ptr[s]; k < S->child_ptr[s + 1]; ++k) {
            int c = S->child[k];
            int64_t o = S->upd_off[c];
            for (int64_t t = S->row_ptr[c] + S->sn_ncol[c]; t < S->row_ptr[c + 1]; ++t)
                S->rel[o++] = pos[S->rows[t]];
        }
        // assembly map for this supernode's columns
        int first = S->sn_first[s], last = S->sn_first[s + 1] - 1;
        int f = S->sn_nrow[s];
        for (int j = first; j <= last; ++j) {
            int o = perm[j];
            for (int64_t t = K.rowptr[o]; t < K.rowptr[o + 1]; ++t) {
                int i = ip[K.colidx[t]];
                if (i < j) continue;
                S->amap_slot.push_back(t);
                S->amap_off.push_back((int64_t)(j - first) * f + pos[i]);
            }
        }
        S->amap_ptr[s + 1] = (int64_t)S->amap_slot.size();
        for (int64_t t = S->row_ptr[s]; t < S->row_ptr[s + 1]; ++t) pos[S->rows[t]] = -1;
    }
    if (ns == 0) S->amap_ptr.assign(1, 0);
    S->dsign.resize(N);
    for (int j = 0; j < N; ++j) S->dsign[j] = K.sign[perm[j]];
    return used;
}

}  // namespace qoco
