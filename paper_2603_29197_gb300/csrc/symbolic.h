// Host-side set-up of the KKT system: validation, pattern assembly (paper §2.2,
// eq. (2)), fill-reducing ordering and the symbolic supernodal analysis.  The paper
// runs this phase once per problem on the CPU (inside cuDSS's analysis phase, §2.2,
// whose cost dominates its set-up time, §3.2); here it is our own C++ code.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "qoco_gpu.h"

namespace qoco {

// Full symmetric KKT pattern in CSR (row i lists all j with K_ij stored), original
// x | y | z numbering.  Every diagonal slot exists; SOC blocks of −WᵀW are dense.
struct KKTPattern {
    int n = 0, m = 0, p = 0, l = 0, nsoc = 0;
    int N = 0;                          // n + p + m
    std::vector<int> q;                 // SOC dims
    std::vector<int> cone_off;          // start (within z, i.e. 0..m) of each SOC
    std::vector<int64_t> rowptr;        // N + 1
    std::vector<int> colidx;            // nnz
    std::vector<double> val0;           // initial values (P, A, G; zero elsewhere)
    std::vector<int64_t> diag_slot;     // N
    std::vector<int64_t> w2_slot;       // l + Σ q²: orthant diagonals, then each SOC block row-major
    std::vector<int64_t> w2_ptr;        // nsoc + 1 offsets into the SOC part of w2_slot (after l)
    std::vector<signed char> sign;      // +1 for x rows, −1 for y and z rows
    // value sources for parametric updates: slot ← src index into [P.val | A.val | G.val]
    std::vector<int64_t> src;           // nnz, −1 where the slot is not data
    int64_t nnzP = 0, nnzA = 0, nnzG = 0;
    int64_t nnz() const { return (int64_t)colidx.size(); }
};

// Validates the problem data; on failure returns a QOCO_GPU_ERR_* code and fills msg.
int validate_problem(int n, int m, int p, const qoco_csc* P, const double* c,
                     const qoco_csc* A, const double* b, const qoco_csc* G,
                     const double* h, int l, int nsoc, const int* q, bool check_vectors,
                     std::string* msg);

// Builds the KKT pattern; assumes validate_problem succeeded.
void build_kkt_pattern(KKTPattern* K, int n, int m, int p, const qoco_csc* P,
                       const qoco_csc* A, const qoco_csc* G, int l, int nsoc, const int* q);

// Adjacency of the KKT graph without the diagonal (CSR over the N nodes).
struct Graph {
    int N = 0;
    std::vector<int64_t> ptr;
    std::vector<int> adj;
};
Graph kkt_graph(const KKTPattern& K);

// Orderings: perm[new] = old.
std::vector<int> order_amd(const Graph& g, double dense_factor = 10.0);
std::vector<int> order_nd(const Graph& g, int leaf_size);

// Supernodal symbolic factorisation of the permuted KKT matrix.
struct Symbolic {
    int N = 0;
    std::vector<int> perm, iperm;       // perm[new] = old; iperm[old] = new
    // supernodes in topological (postorder) order: children before parents
    int ns = 0;
    std::vector<int> sn_first;          // ns + 1: first column of each supernode
    std::vector<int> sn_ncol;           // c_s
    std::vector<int> sn_nrow;           // f_s = c_s + r_s
    std::vector<int> sn_parent;         // −1 for roots
    std::vector<int64_t> row_ptr;       // ns + 1 into rows
    std::vector<int> rows;              // R_s: sorted permuted row indices (own columns first)
    std::vector<int64_t> front_off;     // ns + 1: Σ f² prefix (doubles)
    std::vector<int64_t> upd_off;       // ns + 1: Σ r prefix (update vectors / relative maps)
    std::vector<int> rel;               // Σ r: position of R_s[c_s + a] inside the parent's R
    std::vector<int> child_ptr, child;  // children lists (CSR over supernodes)
    std::vector<int> level;             // height in the supernodal tree (leaves 0)
    int n_levels = 0;
    std::vector<int> level_ptr, level_list;   // supernodes grouped by level
    // assembly map: KKT lower entries (permuted) of each supernode's columns
    std::vector<int64_t> amap_ptr;      // ns + 1
    std::vector<int64_t> amap_slot;     // slot in the KKT value array
    std::vector<int64_t> amap_off;      // column-major offset inside the front (col·f + row)
    std::vector<signed char> dsign;     // sign of each permuted column
    // statistics
    int64_t l_nnz = 0;                  // Σ c_j (below-diagonal counts)
    double flops = 0.0;                 // Σ c_j² + 2 c_j
    int max_front = 0;
    int64_t front_entries = 0;
};

// Column counts and etree statistics of a candidate ordering (cheap, used by AUTO).
struct OrderingCost {
    double flops = 0.0;
    int64_t l_nnz = 0;
    int height = 0;
};
OrderingCost ordering_cost(const KKTPattern& K, const std::vector<int>& perm);

// ND's leaf size for a graph of N nodes: the setting, or when it is ≤ 0 an automatic
// size from N.
int nd_leaf_size(const qoco_gpu_settings& st, int N);

// AUTO's choice between an AMD and an ND candidate of the same matrix or batch (`trees`
// independent problems): true when the ND candidate is cheaper by the cost model.
bool auto_picks_nd(const OrderingCost& amd, const OrderingCost& nd, const qoco_gpu_settings& st, int trees);

// Orderings of a batch whose instances fall into a few distinct sparsity patterns
// (count[c] instances share pats[c]): each pattern is ordered once, by AMD, ND or, for
// AUTO, both, the choice made on the batch's totals (flops add over the instances, the
// tree height is the tallest instance's).  perms[c] is pattern c's ordering (new → old,
// in the pattern's own numbering).  Returns the ordering used.
int order_batch_patterns(const std::vector<KKTPattern>& pats, const std::vector<int>& count,
                         const qoco_gpu_settings& st, int trees, std::vector<std::vector<int>>* perms);

// Where each instance of a batch sits in the block-diagonal stack: its x rows, y rows,
// orthant rows and SOC rows (prefix offsets over the instances, nb + 1 entries each; the
// stack's rows are all x, then all y, then every orthant row, then every SOC row), its
// SOCs, and the first entry of its data in the stack's P, A and G value arrays.
struct StackLayout {
    int n = 0, p = 0, m = 0, l = 0;
    std::vector<int> xo, yo, lo, so, ko;
    std::vector<int64_t> Poff, Aoff, Goff;  // nb + 1 each
    int nb() const { return (int)xo.size() - 1; }
    // stack row of instance i's local KKT row o (local numbering x | y | z, z = orthant
    // rows then SOC rows)
    int row(int i, int o) const {
        const int ni = xo[i + 1] - xo[i], pi = yo[i + 1] - yo[i], li = lo[i + 1] - lo[i];
        if (o < ni) return xo[i] + o;
        if (o < ni + pi) return n + yo[i] + (o - ni);
        const int r = o - ni - pi;
        return n + p + (r < li ? lo[i] + r : l + so[i] + (r - li));
    }
};

// The KKT pattern and analysis of a block-diagonal stack assembled from each distinct
// instance pattern's own (pats[c], syms[c]; instance i has pattern cls[i]) by mapping
// rows, columns, supernodes and value slots to the stack: the result equals what
// build_kkt_pattern and analyze give on the stack with the instances' orderings
// concatenated (an elimination forest is postordered tree by tree, and amalgamation and
// absorption never cross trees).  q: the stack's SOC dimensions; Pv, Av, Gv: the stack's
// data values.  Runs on a few host threads over the instances.
void stack_analysis(const std::vector<KKTPattern>& pats, const std::vector<Symbolic>& syms,
                    const std::vector<int>& cls, const StackLayout& L, const std::vector<int>& q,
                    const double* Pv, const double* Av, const double* Gv, KKTPattern* K, Symbolic* S);

// Full analysis for a given ordering choice; returns the ordering actually used.
// `trees` is the number of independent problems stacked in K (a batch): their chains
// of dependent fronts run side by side, which AUTO's cost model takes into account.
// With perm0 the ordering step is skipped: perm0 (new → old) is used as the fill-
// reducing ordering and perm0_ordering is reported as the ordering used.
int analyze(const KKTPattern& K, const qoco_gpu_settings& st, Symbolic* S, int trees = 1,
            const std::vector<int>* perm0 = nullptr, int perm0_ordering = 0);

}  // namespace qoco
