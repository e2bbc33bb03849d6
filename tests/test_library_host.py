"""CPU tests of the C-ABI library: it loads without a GPU, exports every function
that include/qoco_gpu.h declares, validates problem data on the host, and its
host-side symbolic analysis (ordering, column counts, supernodes) agrees with a
brute-force symbolic elimination."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import paper_2603_29197_gb300 as q
from paper_2603_29197_gb300 import _lib
from workloads import Problem, dense_qp, mpc_batch, portfolio_socp, trajectory_socp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "qoco_gpu.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(qoco_gpu_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    assert len(names) >= 15
    for nm in names:
        assert hasattr(lib, nm), nm
        assert nm in _lib.SIGNATURES, f"{nm} missing from the binding"
    assert set(_lib.SIGNATURES) == names


def test_default_settings(lib):
    st = q.default_settings()
    assert st.abstol == 1e-7 and st.reltol == 1e-7
    assert st.max_iter == 200 and st.static_reg == 1e-8 and st.step_fraction == 0.99
    assert st.max_refine == 10 and st.refine_tol == 1e-10
    assert st.mixed_precision == 0 and st.batch_schedule == 0
    assert st.nd_leaf == 0  # automatic


def test_nd_leaf_is_automatic_by_size(lib):
    # N_K / 2048 clamped to 64..256: a 20000-stage trajectory (540k KKT rows) gets leaves
    # of 256, an MPC instance of horizon 60 (1260 rows) leaves of 64
    big = trajectory_socp(N=20000)
    assert np.array_equal(q.analyze(big, ordering=2)[1], q.analyze(big, ordering=2, nd_leaf=256)[1])
    small = mpc_batch(count=1, tmin=60, tmax=60)[0]
    assert np.array_equal(q.analyze(small, ordering=2)[1], q.analyze(small, ordering=2, nd_leaf=64)[1])


def _header_struct(name):
    txt = open(os.path.join(ROOT, "include", "qoco_gpu.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", txt).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(double|int64_t|int|char)\s+(.*)$", decl, flags=re.S)
        ctype, names = m.group(1), m.group(2)
        for nm in names.split(","):
            nm = nm.strip()
            arr = re.match(r"(\w+)\[(\w+)\]", nm)
            fields.append((arr.group(1), ctype, int(arr.group(2))) if arr else (nm, ctype, 1))
    return fields


@pytest.mark.parametrize("cname,pyname", [("qoco_gpu_settings", "Settings"), ("qoco_gpu_info", "Info")])
def test_binding_structs_mirror_the_header(cname, pyname):
    import ctypes as C
    want = {"double": C.c_double, "int": C.c_int, "int64_t": C.c_int64, "char": C.c_char}
    hdr = _header_struct(cname)
    py = getattr(_lib, pyname)._fields_
    assert [f[0] for f in hdr] == [f[0] for f in py]
    for (nm, ctype, n), (_, pytype) in zip(hdr, py):
        assert C.sizeof(pytype) == C.sizeof(want[ctype]) * n, nm


def test_batch_csc_table_reads_back_through_ctypes():
    # the batch binding fills its qoco_csc tables as numpy records of addresses
    import ctypes as C
    from paper_2603_29197_gb300 import _CSC_DTYPE, _csc_row
    tab = np.zeros(3, dtype=_CSC_DTYPE)
    M = sp.random(7, 5, density=0.4, format="csc", random_state=1)
    keep = _csc_row(tab, 1, M, 7, 5)
    ptr = tab.ctypes.data_as(C.POINTER(_lib.CSC))
    assert ptr[0].colptr is None or not bool(ptr[0].colptr)  # untouched rows stay NULL
    got = ptr[1]
    assert (got.n_rows, got.n_cols, got.nnz) == (7, 5, M.nnz)
    assert [got.colptr[j] for j in range(6)] == list(M.indptr)
    assert [got.rowidx[t] for t in range(M.nnz)] == list(M.indices)
    assert [got.val[t] for t in range(M.nnz)] == list(M.data)
    del keep


def _tiny(**kw):
    P = sp.csc_matrix(np.array([[2.0, 0.5], [0.0, 1.0]]))
    A = sp.csc_matrix(np.array([[1.0, 1.0]]))
    G = sp.csc_matrix(np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]]))
    d = dict(n=2, m=3, p=1, P=P, c=np.zeros(2), A=A, b=np.ones(1), G=G, h=np.ones(3), l=1, q=[2])
    d.update(kw)
    return Problem(**d)


@pytest.mark.parametrize("mut,code", [
    (dict(l=2), _lib.ERR_INVALID_CONE),                      # l + Σq ≠ m
    (dict(q=[1, 1], l=1), _lib.ERR_INVALID_CONE),            # SOC of dimension 1
    (dict(P=sp.csc_matrix(np.array([[2.0, 0.0], [0.5, 1.0]]))), _lib.ERR_INVALID_CSC),  # lower P
    (dict(G=sp.csc_matrix(np.ones((2, 2)))), _lib.ERR_INVALID_DIMS),
    (dict(A=sp.csc_matrix(np.array([[np.nan, 1.0]]))), _lib.ERR_NONFINITE_DATA),
])
def test_host_validation(lib, mut, code):
    with pytest.raises(ValueError) as e:
        q.analyze(_tiny(**mut))
    assert _lib.STATUS_NAMES[code] in str(e.value)


def test_unsorted_rows_rejected(lib):
    pr = _tiny()
    G = pr.G.copy()
    G.indices = G.indices.copy()
    # column 0 has rows [0, 2]; swap them
    G.indices[0], G.indices[1] = G.indices[1], G.indices[0]
    pr.G = G
    with pytest.raises(ValueError, match="invalid_csc"):
        q.analyze(pr)


def _kkt_pattern(prob):
    n, p, m = prob.n, prob.p, prob.m
    N = n + p + m
    Pu = prob.P.toarray() != 0
    B = np.zeros((N, N), dtype=bool)
    B[:n, :n] = Pu | Pu.T
    B[n:n + p, :n] = prob.A.toarray() != 0
    B[n + p:, :n] = prob.G.toarray() != 0
    B = B | B.T
    o = n + p + prob.l
    for qk in prob.q:
        B[o:o + qk, o:o + qk] = True
        o += qk
    np.fill_diagonal(B, True)
    return B


def _symbolic_counts(B):
    """Below-diagonal counts of L by explicit boolean elimination."""
    B = B.copy()
    N = B.shape[0]
    counts = np.zeros(N, dtype=np.int64)
    for j in range(N):
        below = np.nonzero(B[j + 1:, j])[0] + j + 1
        counts[j] = below.size
        if below.size:
            B[np.ix_(below, below)] = True
    return counts


@pytest.mark.parametrize("make", [lambda: dense_qp(n=40, p=8, m=60, rank=5, density=0.1, seed=3),
                                  lambda: trajectory_socp(N=30, seed=1),
                                  lambda: portfolio_socp(n=60, k=6, seed=2)],
                         ids=["dense_qp", "trajectory", "portfolio"])
@pytest.mark.parametrize("order", [q.ORDER_AMD, q.ORDER_ND, q.ORDER_NATURAL, q.ORDER_AUTO])
def test_symbolic_counts_match_brute_force(lib, make, order):
    prob = make()
    info, perm, sn = q.analyze(prob, ordering=order, nd_leaf=16)
    N = prob.n + prob.p + prob.m
    assert sorted(perm.tolist()) == list(range(N))
    B = _kkt_pattern(prob)[np.ix_(perm, perm)]
    cnt = _symbolic_counts(B)
    assert info["l_nnz"] == cnt.sum()
    assert np.isclose(info["factor_flops"], float(np.sum(cnt.astype(float) ** 2 + 2 * cnt)))
    assert sn[0] == 0 and sn[-1] == N and np.all(np.diff(sn) > 0)
    assert info["kkt_nnz"] == B.sum()
    if order == q.ORDER_NATURAL:
        np.testing.assert_array_equal(perm, np.arange(N))


def test_nested_dissection_gives_shallow_tree_on_stage_chains(lib):
    prob = trajectory_socp(N=2000)
    i_amd, _, _ = q.analyze(prob, ordering=q.ORDER_AMD)
    i_nd, _, _ = q.analyze(prob, ordering=q.ORDER_ND)
    i_auto, _, _ = q.analyze(prob)
    assert i_nd["n_levels"] <= 30 < i_amd["n_levels"]
    assert i_auto["ordering_used"] == q.ORDER_ND


def test_amd_orders_dense_rows_last(lib):
    prob = portfolio_socp(n=2000, k=40, seed=1)
    info, perm, _ = q.analyze(prob, ordering=q.ORDER_AMD)
    # the budget row and the risk-cone rows Fᵀx couple every asset: they end up last
    n, p = prob.n, prob.p
    core = {n} | set(range(n + p + prob.l + 1, n + p + prob.m))
    assert set(perm[-len(core):].tolist()) == core
    assert info["n_levels"] <= 4


def test_nested_dissection_is_reproducible_across_host_threads(lib):
    # 135k KKT nodes: the top separators' parts are dissected on concurrent host threads;
    # the order must not depend on their timing
    pr = trajectory_socp(N=5000, seed=4)
    perms = [q.analyze(pr, ordering=2)[1] for _ in range(3)]
    assert all(np.array_equal(perms[0], p) for p in perms[1:])
    assert sorted(perms[0].tolist()) == list(range(len(perms[0])))


def _stack(probs):
    # block-diagonal stack with every orthant row first, then every SOC row
    P = sp.block_diag([sp.csc_matrix(p.P) for p in probs], format="csc")
    A = sp.block_diag([sp.csc_matrix(p.A) for p in probs], format="csc")
    G = sp.vstack([sp.block_diag([sp.csc_matrix(p.G)[:p.l] for p in probs]),
                   sp.block_diag([sp.csc_matrix(p.G)[p.l:] for p in probs])]).tocsc()
    return Problem(n=P.shape[0], m=G.shape[0], p=A.shape[0], P=P, c=np.zeros(P.shape[0]), A=A,
                   b=np.zeros(A.shape[0]), G=G, h=np.zeros(G.shape[0]), l=sum(p.l for p in probs),
                   q=sum([list(p.q) for p in probs], []))


def test_nested_dissection_of_many_components_is_reproducible(lib):
    # 96 independent MPC instances (~70k KKT nodes): the components are dissected on
    # concurrent host threads in contiguous ranges; the order is the component order
    pr = _stack(mpc_batch(count=96, tmin=10, tmax=60, seed=5))
    perms = [q.analyze(pr, ordering=2)[1] for _ in range(3)]
    assert all(np.array_equal(perms[0], p) for p in perms[1:])
    assert sorted(perms[0].tolist()) == list(range(len(perms[0])))


def _stack_rows(probs):
    """Stack row of every instance's local KKT row (x | y | z, z = orthant then SOC rows),
    in the block-diagonal layout qoco_gpu_setup_batch uses."""
    nt, pt, lt = (sum(int(getattr(pr, k)) for pr in probs) for k in ("n", "p", "l"))
    xo = yo = lo = so = 0
    out = []
    for pr in probs:
        n, p, m, l = int(pr.n), int(pr.p), int(pr.m), int(pr.l)
        r = np.arange(m)
        z = np.where(r < l, nt + pt + lo + r, nt + pt + lt + so + (r - l))
        out.append(np.concatenate([xo + np.arange(n), nt + yo + np.arange(p), z]))
        xo, yo, lo, so = xo + n, yo + p, lo + l, so + (m - l)
    return out


@pytest.mark.parametrize("order", [1, 2])
def test_batch_analysis_is_the_instances_analyses_stacked(lib, order):
    # repeated MPC patterns (horizons 10..13) with other models between them: the batch's
    # ordering, supernodes, front orders and levels are each instance's own, relabelled
    probs = mpc_batch(count=20, tmin=10, tmax=13, seed=5)
    probs = probs[:9] + [dense_qp(n=40, p=8, m=60, rank=6, density=0.1, seed=22),
                         portfolio_socp(n=50, k=6, seed=23), trajectory_socp(N=12, seed=6)] + probs[9:]
    info, perm, sn, fs, lv = q.analyze_batch(probs, ordering=order)
    one = [q.analyze(pr, ordering=order, structure=True) for pr in probs]
    assert info["ordering_used"] == order
    for k in ("factor_flops", "l_nnz", "n_supernodes", "kkt_nnz", "kkt_dim", "front_entries"):
        assert info[k] == sum(o[0][k] for o in one), k
    assert info["max_front"] == max(o[0]["max_front"] for o in one)
    assert info["n_levels"] == max(o[0]["n_levels"] for o in one)
    rows = _stack_rows(probs)
    co = so = 0
    for i, (inf, pm, s, f, v) in enumerate(one):
        N, ns = len(pm), inf["n_supernodes"]
        assert np.array_equal(perm[co:co + N], rows[i][pm]), i
        assert np.array_equal(sn[so:so + ns + 1], s + co), i
        assert np.array_equal(fs[so:so + ns], f) and np.array_equal(lv[so:so + ns], v), i
        co, so = co + N, so + ns
    assert co == len(perm) and sn[-1] == co


@pytest.mark.parametrize("order", [1, 2])
def test_batch_analysis_edge_layouts(lib, order):
    # instances without equality rows, without an orthant, without P, and with only an
    # orthant, repeated and interleaved: every branch of the stack's row map
    rng = np.random.default_rng(3)

    def inst(n, p, l, q, with_P=True):
        m = l + sum(q)
        G = sp.csc_matrix(rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.6))
        P = sp.csc_matrix(np.triu(np.eye(n) * 2.0 + 0.1)) if with_P else sp.csc_matrix((n, n))
        A = sp.csc_matrix(rng.standard_normal((p, n))) if p else sp.csc_matrix((0, n))
        for M in (G, P, A):
            M.sort_indices()
        return Problem(n=n, m=m, p=p, P=P, c=rng.standard_normal(n), A=A, b=np.ones(p), G=G,
                       h=np.ones(m), l=l, q=list(q))
    kinds = [(6, 0, 3, [3]), (5, 2, 0, [3, 2]), (4, 1, 4, [], False), (7, 0, 0, [4, 3]), (5, 2, 3, [2])]
    probs = []
    for r in range(3):
        for k in kinds:
            probs.append(inst(*k))
    info, perm, sn, fs, lv = q.analyze_batch(probs, ordering=order)
    one = [q.analyze(pr, ordering=order, structure=True) for pr in probs]
    assert info["factor_flops"] == sum(o[0]["factor_flops"] for o in one)
    assert info["kkt_nnz"] == sum(o[0]["kkt_nnz"] for o in one)
    rows = _stack_rows(probs)
    co = so = 0
    for i, (inf, pm, s, f, v) in enumerate(one):
        N, ns = len(pm), inf["n_supernodes"]
        assert np.array_equal(perm[co:co + N], rows[i][pm]), i
        assert np.array_equal(sn[so:so + ns + 1], s + co) and np.array_equal(fs[so:so + ns], f), i
        co, so = co + N, so + ns


def test_batch_analysis_auto_and_natural(lib):
    probs = mpc_batch(count=24, tmin=10, tmax=30, seed=9)
    auto = q.analyze_batch(probs)[0]
    assert auto["ordering_used"] in (1, 2)
    pick = q.analyze_batch(probs, ordering=auto["ordering_used"])[0]
    assert pick["factor_flops"] == auto["factor_flops"]
    nat = q.analyze_batch(probs, ordering=3)[0]
    assert nat["ordering_used"] == 3 and nat["kkt_nnz"] == auto["kkt_nnz"]
    bad = list(probs)
    bad[5] = _tiny(l=2)
    with pytest.raises(ValueError) as e:
        q.analyze_batch(bad)
    assert "instance 5" in str(e.value)
    # an instance without cone rows has no barrier parameter: rejected by name
    n = 3
    eq = Problem(n=n, m=0, p=1, P=sp.csc_matrix(np.eye(n)), c=np.ones(n), A=sp.csc_matrix(np.ones((1, n))),
                 b=np.ones(1), G=sp.csc_matrix((0, n)), h=np.zeros(0), l=0, q=[])
    with pytest.raises(ValueError) as e:
        q.analyze_batch(probs[:2] + [eq] + probs[2:])
    assert "instance 2" in str(e.value) and "cone rows" in str(e.value)
    assert _lib.STATUS_NAMES[_lib.ERR_NOT_IMPLEMENTED] in str(e.value)
