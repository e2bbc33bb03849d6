// Fill-reducing orderings of the KKT graph, run once at set-up.
//
//  * order_amd: approximate minimum degree on the quotient graph (Amestoy, Davis &
//    Duff, SIAM J. Matrix Anal. Appl. 17(4), 1996): eliminated nodes become elements,
//    degrees are the approximate external degrees of that paper's bound, elements
//    that become subsets of the new element are absorbed, indistinguishable
//    variables are merged into supervariables (hash + exact comparison), and rows
//    denser than dense_factor·√N are ordered last.  Written from the paper's
//    description with per-node std::vector lists instead of one packed workspace.
//  * order_nd: nested dissection by breadth-first level structures from a
//    pseudo-peripheral node (George & Liu): a level that is small and splits the nodes
//    evenly (least size × larger side, each side ≥ 20%), thinned to the nodes touching
//    the next level, is the vertex separator; parts are dissected recursively and
//    ordered before their separator;
//    parts at or below `leaf_size` nodes (or without a usable separator) are ordered
//    by AMD.  Gives the O(log N)-deep elimination trees that level-scheduled GPU
//    factorisation needs on banded / stage-structured problems.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <functional>
#include <memory>
#include <numeric>
#include <thread>

#include "symbolic.h"

namespace qoco {

namespace {

enum : signed char { VAR = 0, ELEM = 1, DEAD = 2, DENSE = 3 };

}  // namespace

std::vector<int> order_amd(const Graph& g, double dense_factor) {
    const int N = g.N;
    std::vector<int> order;
    order.reserve(N);
    if (N == 0) return order;
    int dense_thr = std::max(16, (int)(dense_factor * std::sqrt((double)N)));
    std::vector<signed char> status(N, VAR);
    int ndense = 0;
    for (int i = 0; i < N; ++i)
        if (N >= 1000 && g.ptr[i + 1] - g.ptr[i] > dense_thr) { status[i] = DENSE; ++ndense; }

    std::vector<std::vector<int>> vars(N), elems(N), Le(N);
    std::vector<int> nv(N, 1), deg(N, 0), wdeg(N, 0), w(N, 0);
    std::vector<int> flag(N, 0), wflag(N, 0), merged_into(N, -1);
    std::vector<uint64_t> hsh(N, 0);
    for (int i = 0; i < N; ++i) {
        if (status[i] == DENSE) continue;
        vars[i].reserve(g.ptr[i + 1] - g.ptr[i]);
        for (int64_t t = g.ptr[i]; t < g.ptr[i + 1]; ++t)
            if (status[g.adj[t]] != DENSE) vars[i].push_back(g.adj[t]);
        deg[i] = (int)vars[i].size();
    }
    std::vector<int> head(N + 1, -1), nxt(N, -1), prv(N, -1);
    int mindeg = N;
    auto insert = [&](int i) {
        int d = deg[i];
        nxt[i] = head[d];
        prv[i] = -1;
        if (head[d] >= 0) prv[head[d]] = i;
        head[d] = i;
        if (d < mindeg) mindeg = d;
    };
    auto remove = [&](int i) {
        if (prv[i] >= 0) nxt[prv[i]] = nxt[i];
        else head[deg[i]] = nxt[i];
        if (nxt[i] >= 0) prv[nxt[i]] = prv[i];
    };
    int nleft = 0;
    for (int i = 0; i < N; ++i)
        if (status[i] == VAR) { insert(i); ++nleft; }

    int stamp = 0;
    std::vector<int> Lp;
    std::vector<int> tmpE, tmpV, tmpE2, tmpV2;
    while (nleft > 0) {
        while (mindeg <= N && head[mindeg] < 0) ++mindeg;
        const int p = head[mindeg];
        remove(p);
        ++stamp;
        Lp.clear();
        flag[p] = stamp;
        for (int e : elems[p]) {
            if (status[e] != ELEM) continue;
            for (int i : Le[e])
                if (status[i] == VAR && flag[i] != stamp) { flag[i] = stamp; Lp.push_back(i); }
            status[e] = DEAD;  // absorbed into the new element p
            std::vector<int>().swap(Le[e]);
        }
        for (int i : vars[p])
            if (status[i] == VAR && flag[i] != stamp) { flag[i] = stamp; Lp.push_back(i); }
        status[p] = ELEM;
        std::vector<int>().swap(vars[p]);
        std::vector<int>().swap(elems[p]);
        order.push_back(p);
        nleft -= nv[p];

        int degLp = 0;
        for (int i : Lp) degLp += nv[i];
        // |Le \ Lp| for every element adjacent to Lp
        for (int i : Lp) {
            remove(i);
            for (int e : elems[i]) {
                if (status[e] != ELEM) continue;
                if (wflag[e] != stamp) { wflag[e] = stamp; w[e] = wdeg[e] - nv[i]; }
                else w[e] -= nv[i];
            }
        }
        // degree update, list pruning, aggressive absorption
        for (int i : Lp) {
            // both lists filtered in place (order kept), p appended to the elements
            std::vector<int>& Ei = elems[i];
            size_t ke = 0;
            int dext = 0;
            for (size_t x = 0; x < Ei.size(); ++x) {
                const int e = Ei[x];
                if (status[e] != ELEM) continue;
                if (w[e] <= 0) {  // Le ⊆ Lp: absorb e into p
                    status[e] = DEAD;
                    std::vector<int>().swap(Le[e]);
                    continue;
                }
                Ei[ke++] = e;
                dext += w[e];
            }
            Ei.resize(ke);
            Ei.push_back(p);
            std::vector<int>& Vi = vars[i];
            size_t kv = 0;
            int dv = 0;
            for (size_t x = 0; x < Vi.size(); ++x) {
                const int j = Vi[x];
                if (status[j] == VAR && flag[j] != stamp) { Vi[kv++] = j; dv += nv[j]; }
            }
            Vi.resize(kv);
            long d1 = (long)dv + degLp - nv[i] + dext;
            long d2 = (long)deg[i] + degLp - nv[i];
            long d3 = (long)nleft - nv[i];
            long d = std::min(d1, std::min(d2, d3));
            deg[i] = (int)std::max(0L, d);
            uint64_t hv = 0;
            for (int e : elems[i]) hv += (uint64_t)e * 0x9E3779B97F4A7C15ull + 1;
            for (int j : vars[i]) hv += (uint64_t)j * 0xC2B2AE3D27D4EB4Full + 7;
            hsh[i] = hv;
        }
        // supervariable detection among Lp
        if (Lp.size() > 1) {
            std::vector<int> idx(Lp);
            std::sort(idx.begin(), idx.end(), [&](int a, int b) {
                if (hsh[a] != hsh[b]) return hsh[a] < hsh[b];
                return a < b;
            });
            for (size_t a = 0; a < idx.size();) {
                size_t b = a + 1;
                while (b < idx.size() && hsh[idx[b]] == hsh[idx[a]]) ++b;
                if (b - a > 1) {
                    for (size_t x = a; x < b; ++x) {
                        int i = idx[x];
                        if (status[i] != VAR) continue;
                        tmpE = elems[i]; std::sort(tmpE.begin(), tmpE.end());
                        tmpV = vars[i]; std::sort(tmpV.begin(), tmpV.end());
                        for (size_t y = x + 1; y < b; ++y) {
                            int j = idx[y];
                            if (status[j] != VAR) continue;
                            if (elems[j].size() != tmpE.size() || vars[j].size() != tmpV.size()) continue;
                            tmpE2 = elems[j]; std::sort(tmpE2.begin(), tmpE2.end());
                            if (tmpE2 != tmpE) continue;
                            tmpV2 = vars[j]; std::sort(tmpV2.begin(), tmpV2.end());
                            if (tmpV2 != tmpV) continue;
                            // merge j into i
                            nv[i] += nv[j];
                            deg[i] = std::max(0, deg[i] - nv[j]);
                            nv[j] = 0;
                            status[j] = DEAD;
                            merged_into[j] = i;
                            std::vector<int>().swap(vars[j]);
                            std::vector<int>().swap(elems[j]);
                        }
                    }
                }
                a = b;
            }
        }
        // the new element and the reinsertion of its variables
        std::vector<int>& L = Le[p];
        L.clear();
        int wsum = 0;
        for (int i : Lp)
            if (status[i] == VAR) { L.push_back(i); wsum += nv[i]; }
        wdeg[p] = wsum;
        for (int i : L) {
            deg[i] = std::min(deg[i], std::max(0, nleft - nv[i]));
            insert(i);
        }
    }

    // expand supervariables: each eliminated principal is followed by its members
    // (member lists in increasing index order, as singly linked lists with a tail)
    std::vector<int> mhead(N, -1), mtail(N, -1), mnext(N, -1);
    for (int j = 0; j < N; ++j) {
        const int r = merged_into[j];
        if (r < 0) continue;
        if (mtail[r] < 0) mhead[r] = j;
        else mnext[mtail[r]] = j;
        mtail[r] = j;
    }
    std::vector<int> out;
    out.reserve(N);
    std::vector<int> stack;
    for (int p : order) {
        stack.assign(1, p);
        while (!stack.empty()) {
            int v = stack.back();
            stack.pop_back();
            out.push_back(v);
            for (int u = mhead[v]; u >= 0; u = mnext[u]) stack.push_back(u);
        }
    }
    for (int i = 0; i < N; ++i)
        if (status[i] == DENSE) out.push_back(i);
    return out;
}

namespace {

// Shared marks of the dissection.  Subproblems that run concurrently own disjoint node
// sets; a node's tag is written only by the subproblem that owns it, but a BFS reads the
// tags of its nodes' neighbours, which may belong to a concurrent subproblem, so tags are
// atomics (relaxed: a foreign tag is never equal to the reader's own).  Levels and local
// indices are read and written only for a subproblem's own nodes.
struct Marks {
    explicit Marks(int n) : tag(new std::atomic<int>[n]), lev(n, -1), local(n, -1) {
        for (int i = 0; i < n; ++i) tag[i].store(0, std::memory_order_relaxed);
    }
    std::unique_ptr<std::atomic<int>[]> tag;
    std::vector<int> lev, local;
    std::atomic<int> next_tag{1};
    int get(int v) const { return tag[v].load(std::memory_order_relaxed); }
    void set(int v, int t) { tag[v].store(t, std::memory_order_relaxed); }
};

// AMD on the subgraph induced by `nodes` (all tagged t); appends the ordered nodes to `out`.
void amd_subset(const Graph& g, Marks& mk, int t, const std::vector<int>& nodes, std::vector<int>* out) {
    const int n = (int)nodes.size();
    if (n <= 2) {
        out->insert(out->end(), nodes.begin(), nodes.end());
        return;
    }
    for (int i = 0; i < n; ++i) mk.local[nodes[i]] = i;
    Graph sg;
    sg.N = n;
    sg.ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        int v = nodes[i];
        for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
            int u = g.adj[e];
            if (mk.get(u) == t) sg.adj.push_back(mk.local[u]);
        }
        sg.ptr[i + 1] = (int64_t)sg.adj.size();
    }
    std::vector<int> o = order_amd(sg);
    for (int i : o) out->push_back(nodes[i]);
    for (int i = 0; i < n; ++i) mk.local[nodes[i]] = -1;
}

// Subproblems at least this large are split across two host threads (the first part on
// a new thread) while fewer than kNdMaxDepth splits are in flight above them; the
// order produced is the serial one (each part's order is computed independently and
// the parts are concatenated in the serial order).
constexpr int kNdParallelMin = 20000;
constexpr int kNdMaxDepth = 4;

struct ND {
    const Graph& g;
    Marks& mk;
    int leaf;
    std::vector<int> q;  // BFS queue (per ND object: one per host thread)

    ND(const Graph& gg, Marks& m, int leaf_size) : g(gg), mk(m), leaf(leaf_size) {}

    // BFS within the nodes carrying tag t; returns levels (as offsets into q).
    int bfs(int root, int t, std::vector<int>& lptr) {
        std::vector<int>& lev = mk.lev;
        q.clear();
        lptr.clear();
        q.push_back(root);
        lev[root] = 0;
        size_t h = 0;
        lptr.push_back(0);
        int cur = 0;
        while (h < q.size()) {
            int v = q[h];
            if (lev[v] != cur) { lptr.push_back((int)h); cur = lev[v]; }
            ++h;
            for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; ++e) {
                int u = g.adj[e];
                if (mk.get(u) == t && lev[u] < 0) { lev[u] = lev[v] + 1; q.push_back(u); }
            }
        }
        lptr.push_back((int)q.size());
        return (int)lptr.size() - 1;  // number of levels
    }
    void clear_lev() { for (int v : q) mk.lev[v] = -1; }

    int local_degree(int v, int t) const {
        int d = 0;
        for (int64_t e = g.ptr[v]; e < g.ptr[v + 1]; ++e) d += mk.get(g.adj[e]) == t;
        return d;
    }

    void leaf_amd(const std::vector<int>& nodes, std::vector<int>* out) {
        const int t = mk.next_tag.fetch_add(1, std::memory_order_relaxed);
        for (int v : nodes) mk.set(v, t);
        amd_subset(g, mk, t, nodes, out);
    }

    // Independent components (a batch's instances, or a part that a separator split) in
    // their order; large sets of them are split into contiguous ranges of about equal
    // node counts, one host thread per range, and the ranges' orders are concatenated in
    // component order.  hint0: a starting node for the first component (see run), or −1.
    void run_components(std::vector<std::vector<int>>& comps, std::vector<int>* out, int depth, int hint0) {
        int64_t total = 0;
        for (const auto& c : comps) total += (int64_t)c.size();
        const int hw = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        const int nth = (int)std::min<int64_t>(hw, (int64_t)comps.size());
        if (depth >= kNdMaxDepth || total < kNdParallelMin || nth < 2) {
            for (size_t k = 0; k < comps.size(); ++k) run(std::move(comps[k]), out, depth, k ? -1 : hint0);
            return;
        }
        std::vector<size_t> cut(1, 0);
        int64_t acc = 0;
        for (size_t k = 0; k < comps.size(); ++k) {
            acc += (int64_t)comps[k].size();
            if ((int)cut.size() < nth && acc * nth >= total * (int64_t)cut.size()) cut.push_back(k + 1);
        }
        if (cut.back() != comps.size()) cut.push_back(comps.size());
        const int nr = (int)cut.size() - 1;
        std::vector<std::vector<int>> outs(nr);
        std::vector<std::thread> ths;
        for (int r = 1; r < nr; ++r)
            ths.emplace_back([this, &comps, &outs, &cut, r]() {
                ND sub(g, mk, leaf);
                for (size_t k = cut[r]; k < cut[r + 1]; ++k) sub.run(std::move(comps[k]), &outs[r], kNdMaxDepth);
            });
        for (size_t k = cut[0]; k < cut[1]; ++k) run(std::move(comps[k]), &outs[0], kNdMaxDepth, k ? -1 : hint0);
        for (auto& t : ths) t.join();
        for (const auto& o : outs) out->insert(out->end(), o.begin(), o.end());
    }

    // hint: a node of `nodes` at an end of the parent's level structure (the parent's BFS
    // root for the first part, its last node for the second), or −1
    void run(std::vector<int> nodes, std::vector<int>* out, int depth, int hint = -1) {
        std::vector<int>& lev = mk.lev;
        if ((int)nodes.size() <= leaf) { leaf_amd(nodes, out); return; }
        const int t = mk.next_tag.fetch_add(1, std::memory_order_relaxed);
        for (int v : nodes) mk.set(v, t);
        // connected components; the first BFS (from nodes[0]) is also the first level
        // structure of the pseudo-peripheral search when the subgraph is connected
        std::vector<int> lptr;
        int nl = bfs(hint >= 0 ? hint : nodes[0], t, lptr);
        if ((int)q.size() < (int)nodes.size()) {
            std::vector<std::vector<int>> comps;
            std::vector<int> seen(q.begin(), q.end());
            comps.emplace_back(q.begin(), q.end());
            for (int v : nodes) {
                if (lev[v] >= 0) continue;
                bfs(v, t, lptr);
                comps.emplace_back(q.begin(), q.end());
                // keep lev marks until all components found
                seen.insert(seen.end(), q.begin(), q.end());
            }
            for (int v : seen) lev[v] = -1;
            // the first component is the hint's: it keeps the hint as its start
            run_components(comps, out, depth, hint);
            return;
        }
        // pseudo-peripheral root: BFS from the least-degree node of the last level while
        // that deepens the level structure; the kept structure is restored from its
        // saved queue instead of a repeated BFS.  A part that starts from the end of its
        // parent's level structure keeps that first structure: the end is already far from
        // the rest of the part (on stage-structured problems it is one end of the part's
        // chain), and the search would cost about two more BFS passes per part.
        std::vector<int> keep_q, keep_l;
        for (int it = 0; it < (hint >= 0 ? 0 : 8); ++it) {
            int best = -1, bd = 1 << 30;
            for (int k = lptr[nl - 1]; k < lptr[nl]; ++k) {
                int d = local_degree(q[k], t);
                if (d < bd) { bd = d; best = q[k]; }
            }
            keep_q.swap(q);
            keep_l.swap(lptr);
            for (int v : keep_q) lev[v] = -1;
            int nl2 = bfs(best, t, lptr);
            if (nl2 <= nl) {
                clear_lev();
                q.swap(keep_q);
                lptr.swap(keep_l);
                for (int k = 0; k < nl; ++k)
                    for (int j = lptr[k]; j < lptr[k + 1]; ++j) lev[q[j]] = k;
                break;
            }
            nl = nl2;
        }
        const int S = (int)nodes.size();
        if (nl < 3) { clear_lev(); amd_subset(g, mk, t, nodes, out); return; }
        // separator level: among the levels whose both sides hold ≥ 20% of the nodes, the
        // one with the least size × larger side (a small separator, and balanced parts:
        // on a chain of equal levels that is the middle one, and the dissection tree stays
        // log₂-deep instead of peeling 20% per level); else the median level
        int pick = -1, median = -1;
        double pcost = 0.0;
        for (int k = 1; k < nl - 1; ++k) {
            int before = lptr[k], after = S - lptr[k + 1];
            int sz = lptr[k + 1] - lptr[k];
            if (median < 0 && lptr[k + 1] >= S / 2) median = k;
            const double cost = (double)sz * std::max(before, after);
            if (before >= S / 5 && after >= S / 5 && (pick < 0 || cost < pcost)) { pcost = cost; pick = k; }
        }
        if (pick < 0) pick = median < 0 ? nl / 2 : median;
        // thin the separator: keep only level nodes touching the next level
        const int hint1 = q[0], hint2 = q[S - 1];  // the ends of this level structure
        std::vector<int> part1, part2, sep;
        part1.reserve(lptr[pick + 1]);
        part2.reserve(S - lptr[pick + 1]);
        for (int k = 0; k < lptr[pick]; ++k) part1.push_back(q[k]);
        for (int k = lptr[pick + 1]; k < S; ++k) part2.push_back(q[k]);
        for (int k = lptr[pick]; k < lptr[pick + 1]; ++k) {
            int v = q[k];
            bool touches = false;
            for (int64_t e = g.ptr[v]; e < g.ptr[v + 1] && !touches; ++e) {
                int u = g.adj[e];
                touches = mk.get(u) == t && lev[u] == pick + 1;
            }
            (touches ? sep : part1).push_back(v);
        }
        clear_lev();
        if ((double)sep.size() > 0.4 * S || part1.empty() || part2.empty()) {
            amd_subset(g, mk, t, nodes, out);
            return;
        }
        // the separator's nodes keep tag t while the parts are dissected (the parts take
        // new tags), so that the separator is ordered by AMD on exactly its own nodes
        if (S >= kNdParallelMin && depth < kNdMaxDepth) {
            std::vector<int> out1;
            std::thread th([this, &part1, &out1, depth, hint1]() {
                ND sub(g, mk, leaf);
                sub.run(std::move(part1), &out1, depth + 1, hint1);
            });
            std::vector<int> out2;
            run(std::move(part2), &out2, depth + 1, hint2);
            th.join();
            out->insert(out->end(), out1.begin(), out1.end());
            out->insert(out->end(), out2.begin(), out2.end());
        } else {
            run(std::move(part1), out, depth + 1, hint1);
            run(std::move(part2), out, depth + 1, hint2);
        }
        amd_subset(g, mk, t, sep, out);
    }
};

}  // namespace

std::vector<int> order_nd(const Graph& g, int leaf_size) {
    std::vector<int> out;
    out.reserve(g.N);
    Marks mk(g.N);
    ND nd(g, mk, std::max(leaf_size, 4));
    std::vector<int> all(g.N);
    std::iota(all.begin(), all.end(), 0);
    nd.run(std::move(all), &out, 0);
    return out;
}

}  // namespace qoco
