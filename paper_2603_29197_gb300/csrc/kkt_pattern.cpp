// Validation of the problem data and assembly of the KKT pattern of eq. (2).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>

#include "symbolic.h"

namespace qoco {

static int check_csc(const qoco_csc* M, int rows, int cols, bool upper, const char* name,
                     std::string* msg) {
    char buf[160];
    if (M->n_rows != rows || M->n_cols != cols || M->nnz < 0) {
        snprintf(buf, sizeof buf, "%s: shape %dx%d (nnz %d), expected %dx%d", name, M->n_rows,
                 M->n_cols, M->nnz, rows, cols);
        *msg = buf;
        return QOCO_GPU_ERR_INVALID_DIMS;
    }
    if (M->nnz > 0 && (!M->colptr || !M->rowidx || !M->val)) {
        snprintf(buf, sizeof buf, "%s: NULL array", name);
        *msg = buf;
        return QOCO_GPU_ERR_INVALID_CSC;
    }
    if (!M->colptr) {
        if (M->nnz == 0) return 0;
    }
    if (M->colptr && (M->colptr[0] != 0 || M->colptr[cols] != M->nnz)) {
        snprintf(buf, sizeof buf, "%s: colptr[0]=%d colptr[n]=%d nnz=%d", name, M->colptr[0],
                 M->colptr[cols], M->nnz);
        *msg = buf;
        return QOCO_GPU_ERR_INVALID_CSC;
    }
    for (int j = 0; M->colptr && j < cols; ++j) {
        int a = M->colptr[j], b = M->colptr[j + 1];
        if (b < a) {
            snprintf(buf, sizeof buf, "%s: colptr decreases at column %d", name, j);
            *msg = buf;
            return QOCO_GPU_ERR_INVALID_CSC;
        }
        for (int k = a; k < b; ++k) {
            int i = M->rowidx[k];
            if (i < 0 || i >= rows || (k > a && i <= M->rowidx[k - 1]) || (upper && i > j)) {
                snprintf(buf, sizeof buf, "%s: bad row index %d in column %d%s", name, i, j,
                         upper && i > j ? " (below the diagonal)" : "");
                *msg = buf;
                return QOCO_GPU_ERR_INVALID_CSC;
            }
            if (!std::isfinite(M->val[k])) {
                snprintf(buf, sizeof buf, "%s: non-finite value at (%d,%d)", name, i, j);
                *msg = buf;
                return QOCO_GPU_ERR_NONFINITE_DATA;
            }
        }
    }
    return 0;
}

static int check_vec(const double* v, int len, const char* name, std::string* msg) {
    if (len > 0 && !v) {
        *msg = std::string(name) + ": NULL vector";
        return QOCO_GPU_ERR_INVALID_ARG;
    }
    for (int i = 0; i < len; ++i)
        if (!std::isfinite(v[i])) {
            *msg = std::string(name) + ": non-finite entry";
            return QOCO_GPU_ERR_NONFINITE_DATA;
        }
    return 0;
}

int validate_problem(int n, int m, int p, const qoco_csc* P, const double* c,
                     const qoco_csc* A, const double* b, const qoco_csc* G,
                     const double* h, int l, int nsoc, const int* q, bool check_vectors,
                     std::string* msg) {
    if (n < 1 || m < 0 || p < 0) {
        *msg = "dimensions must satisfy n >= 1, m >= 0, p >= 0";
        return QOCO_GPU_ERR_INVALID_DIMS;
    }
    if ((int64_t)n + p + m > (int64_t)1 << 30) {
        *msg = "KKT dimension too large";
        return QOCO_GPU_ERR_INVALID_DIMS;
    }
    if (l < 0 || nsoc < 0 || (nsoc > 0 && !q)) {
        *msg = "cone description: l and nsoc must be >= 0 and q given when nsoc > 0";
        return QOCO_GPU_ERR_INVALID_CONE;
    }
    int64_t tot = l;
    for (int k = 0; k < nsoc; ++k) {
        if (q[k] < 2) {
            *msg = "every second-order cone needs dimension >= 2";
            return QOCO_GPU_ERR_INVALID_CONE;
        }
        tot += q[k];
    }
    if (tot != m) {
        *msg = "l + sum(q) must equal m";
        return QOCO_GPU_ERR_INVALID_CONE;
    }
    int rc;
    if (P && (rc = check_csc(P, n, n, true, "P", msg))) return rc;
    if (p > 0 && !A) {
        *msg = "A is required when p > 0";
        return QOCO_GPU_ERR_INVALID_ARG;
    }
    if (A && (rc = check_csc(A, p, n, false, "A", msg))) return rc;
    if (m > 0 && !G) {
        *msg = "G is required when m > 0";
        return QOCO_GPU_ERR_INVALID_ARG;
    }
    if (G && (rc = check_csc(G, m, n, false, "G", msg))) return rc;
    if (check_vectors) {
        if ((rc = check_vec(c, n, "c", msg))) return rc;
        if ((rc = check_vec(b, p, "b", msg))) return rc;
        if ((rc = check_vec(h, m, "h", msg))) return rc;
    }
    return 0;
}

void build_kkt_pattern(KKTPattern* K, int n, int m, int p, const qoco_csc* P,
                       const qoco_csc* A, const qoco_csc* G, int l, int nsoc, const int* q) {
    K->n = n; K->m = m; K->p = p; K->l = l; K->nsoc = nsoc;
    const int N = n + p + m;
    K->N = N;
    K->q.assign(q, q + nsoc);
    K->cone_off.resize(nsoc);
    int o = l;
    for (int k = 0; k < nsoc; ++k) { K->cone_off[k] = o; o += q[k]; }
    if (P && P->nnz == 0) P = nullptr;
    K->nnzP = P ? P->nnz : 0;
    K->nnzA = (A && p > 0) ? A->nnz : 0;
    K->nnzG = (G && m > 0) ? G->nnz : 0;

    // pass 1: row counts
    std::vector<int64_t> cnt(N + 1, 0);
    std::vector<char> pdiag(n, 0);
    if (P)
        for (int j = 0; j < n; ++j)
            for (int k = P->colptr[j]; k < P->colptr[j + 1]; ++k) {
                int i = P->rowidx[k];
                if (i == j) { pdiag[j] = 1; cnt[i]++; }
                else { cnt[i]++; cnt[j]++; }
            }
    for (int j = 0; j < n; ++j) if (!pdiag[j]) cnt[j]++;
    if (K->nnzA)
        for (int j = 0; j < n; ++j)
            for (int k = A->colptr[j]; k < A->colptr[j + 1]; ++k) { cnt[n + A->rowidx[k]]++; cnt[j]++; }
    for (int r = 0; r < p; ++r) cnt[n + r]++;
    if (K->nnzG)
        for (int j = 0; j < n; ++j)
            for (int k = G->colptr[j]; k < G->colptr[j + 1]; ++k) { cnt[n + p + G->rowidx[k]]++; cnt[j]++; }
    for (int i = 0; i < l; ++i) cnt[n + p + i]++;
    for (int k = 0; k < nsoc; ++k)
        for (int a = 0; a < q[k]; ++a) cnt[n + p + K->cone_off[k] + a] += q[k];

    K->rowptr.assign(N + 1, 0);
    for (int i = 0; i < N; ++i) K->rowptr[i + 1] = K->rowptr[i] + cnt[i];
    const int64_t nnz = K->rowptr[N];
    K->colidx.assign(nnz, 0);
    K->src.assign(nnz, -1);
    std::vector<int64_t> fill(K->rowptr.begin(), K->rowptr.end() - 1);
    auto put = [&](int i, int j, int64_t s) {
        int64_t at = fill[i]++;
        K->colidx[at] = j;
        K->src[at] = s;
    };
    if (P)
        for (int j = 0; j < n; ++j)
            for (int k = P->colptr[j]; k < P->colptr[j + 1]; ++k) {
                int i = P->rowidx[k];
                put(i, j, k);
                if (i != j) put(j, i, k);
            }
    for (int j = 0; j < n; ++j) if (!pdiag[j]) put(j, j, -1);
    const int64_t oA = K->nnzP, oG = K->nnzP + K->nnzA;
    if (K->nnzA)
        for (int j = 0; j < n; ++j)
            for (int k = A->colptr[j]; k < A->colptr[j + 1]; ++k) {
                put(n + A->rowidx[k], j, oA + k);
                put(j, n + A->rowidx[k], oA + k);
            }
    for (int r = 0; r < p; ++r) put(n + r, n + r, -1);
    if (K->nnzG)
        for (int j = 0; j < n; ++j)
            for (int k = G->colptr[j]; k < G->colptr[j + 1]; ++k) {
                put(n + p + G->rowidx[k], j, oG + k);
                put(j, n + p + G->rowidx[k], oG + k);
            }
    for (int i = 0; i < l; ++i) put(n + p + i, n + p + i, -1);
    for (int k = 0; k < nsoc; ++k)
        for (int a = 0; a < q[k]; ++a)
            for (int b2 = 0; b2 < q[k]; ++b2)
                put(n + p + K->cone_off[k] + a, n + p + K->cone_off[k] + b2, -1);

    // sort each row by column (carry the source along); most rows arrive sorted (the
    // data's columns are visited in order), and those are left as they are
    std::vector<std::pair<int, int64_t>> tmp;
    for (int i = 0; i < N; ++i) {
        int64_t a = K->rowptr[i], b = K->rowptr[i + 1];
        if (std::is_sorted(K->colidx.begin() + a, K->colidx.begin() + b)) continue;
        tmp.resize(b - a);
        for (int64_t t = a; t < b; ++t) tmp[t - a] = {K->colidx[t], K->src[t]};
        std::sort(tmp.begin(), tmp.end());
        for (int64_t t = a; t < b; ++t) { K->colidx[t] = tmp[t - a].first; K->src[t] = tmp[t - a].second; }
    }
    auto slot_of = [&](int i, int j) -> int64_t {
        const int* base = K->colidx.data();
        const int* lo = base + K->rowptr[i];
        const int* hi = base + K->rowptr[i + 1];
        const int* it = std::lower_bound(lo, hi, j);
        return (it != hi && *it == j) ? (int64_t)(it - base) : -1;
    };
    K->diag_slot.resize(N);
    for (int i = 0; i < N; ++i) K->diag_slot[i] = slot_of(i, i);
    K->w2_slot.clear();
    for (int i = 0; i < l; ++i) K->w2_slot.push_back(K->diag_slot[n + p + i]);
    K->w2_ptr.assign(nsoc + 1, 0);
    for (int k = 0; k < nsoc; ++k) {
        K->w2_ptr[k] = (int64_t)K->w2_slot.size() - l;
        int base = n + p + K->cone_off[k];
        for (int a = 0; a < q[k]; ++a)
            for (int b2 = 0; b2 < q[k]; ++b2) K->w2_slot.push_back(slot_of(base + a, base + b2));
    }
    K->w2_ptr[nsoc] = (int64_t)K->w2_slot.size() - l;
    K->sign.resize(N);
    for (int i = 0; i < N; ++i) K->sign[i] = i < n ? 1 : -1;
    // initial values from the data (the z block is set per iteration)
    K->val0.assign(nnz, 0.0);
    for (int64_t t = 0; t < nnz; ++t) {
        int64_t s = K->src[t];
        if (s < 0) continue;
        if (s < oA) K->val0[t] = P->val[s];
        else if (s < oG) K->val0[t] = A->val[s - oA];
        else K->val0[t] = G->val[s - oG];
    }
}

Graph kkt_graph(const KKTPattern& K) {
    Graph g;
    g.N = K.N;
    g.ptr.assign(K.N + 1, 0);
    g.adj.reserve(K.nnz() - K.N);
    for (int i = 0; i < K.N; ++i) {
        for (int64_t t = K.rowptr[i]; t < K.rowptr[i + 1]; ++t)
            if (K.colidx[t] != i) g.adj.push_back(K.colidx[t]);
        g.ptr[i + 1] = (int64_t)g.adj.size();
    }
    return g;
}

}  // namespace qoco
