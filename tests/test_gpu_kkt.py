"""GPU parity of one KKT system at a shared iterate: the −W² update of the value
array (K1/K2), the numeric LDLᵀ (K5) against the oracle's textbook LDLᵀ in the
natural order, the factor's reconstruction in the analysis' own order, and the
refined solve (K6/K7) against the oracle's solve."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cones as oc
from oracle import kkt as ok
from workloads import dense_qp, portfolio_socp, random_cone_iterate, trajectory_socp

from _gpu_util import assert_certificate, rel_inf

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda()


def N(t):
    return t.detach().cpu().numpy()


SMALL = {
    "dense_qp_n30": lambda: dense_qp(n=30, p=5, m=40, rank=4, density=0.2, seed=1),
    "trajectory_N12": lambda: trajectory_socp(N=12, seed=2),
    "portfolio_n25": lambda: portfolio_socp(n=25, k=4, seed=3),
    "dense_qp_c1": lambda: dense_qp(),
    "portfolio_n300": lambda: portfolio_socp(n=300, k=40, seed=4),
}


def _setup(prob, **kw):
    import paper_2603_29197_gb300 as q
    return q.Solver(prob, **kw)


def _oracle_K(prob, s, z):
    W = oc.NTScaling(s, z, prob.l, prob.q)
    return ok.assemble(prob, ok.z_block(W, prob.m))


@pytest.mark.parametrize("name", list(SMALL) + ["portfolio_n400_wide_cone"])
def test_w2_update_of_kkt_values(name):
    # a Q^91 risk cone (> 64): its −W² block is written by the one-thread-per-entry kernel
    prob = SMALL[name]() if name in SMALL else portfolio_socp(n=400, k=90, seed=8)
    s, z, _, _ = random_cone_iterate(prob.l, prob.q, seed=3, scale_spread=2.0)
    S = _setup(prob)
    S.kkt_factor_at(T(s), T(z))
    rowptr, col, val = S.get_kkt()
    Kg = sp.csr_matrix((val, col, rowptr), shape=(S.N, S.N)).toarray()
    Ko = _oracle_K(prob, s, z).toarray()
    scale = np.maximum(np.abs(Ko), 1e-300)
    diff = np.abs(Kg - Ko)
    assert np.all((diff <= 1e-11 * scale) | (diff <= 1e-13 * np.abs(Ko).max()))


# The trajectory KKT is left out here: its P has a zero diagonal on the controls, so in
# the natural order the first pivots are the static regularisation (1e-8) and later
# pivots lose ~8 digits to cancellation in any LDLᵀ; the comparison would test rounding.
@pytest.mark.parametrize("name", ["dense_qp_n30", "portfolio_n25", "portfolio_n300"])
def test_factor_matches_textbook_ldlt_natural_order(name):
    import paper_2603_29197_gb300 as q
    prob = SMALL[name]()
    s, z, _, _ = random_cone_iterate(prob.l, prob.q, seed=4)
    S = _setup(prob, ordering=q.ORDER_NATURAL)
    S.kkt_factor_at(T(s), T(z))
    perm, L, D = S.factor_dense()
    np.testing.assert_array_equal(perm, np.arange(S.N))
    sg = ok.reg_signs(prob)
    Ke = _oracle_K(prob, s, z).toarray() + 1e-8 * np.diag(sg)
    Lo, Do = ok.dense_ldlt(Ke, signs=sg)
    np.testing.assert_allclose(D, Do, rtol=1e-8)
    assert rel_inf(L, Lo) <= 1e-8


@pytest.mark.parametrize("name", list(SMALL))
def test_factor_reconstructs_permuted_matrix(name):
    prob = SMALL[name]()
    s, z, _, _ = random_cone_iterate(prob.l, prob.q, seed=5, scale_spread=1.0)
    S = _setup(prob)
    S.kkt_factor_at(T(s), T(z))
    perm, L, D = S.factor_dense()
    Ke = (_oracle_K(prob, s, z) + sp.diags(1e-8 * ok.reg_signs(prob))).toarray()
    Kp = Ke[np.ix_(perm, perm)]
    R = (L * D) @ L.T
    assert np.max(np.abs(R - Kp)) <= 1e-11 * np.abs(Kp).max() * max(1.0, np.abs(L).max()) ** 2


@pytest.mark.parametrize("name,spread", [("dense_qp_c1", 0.0), ("trajectory_N12", 3.0),
                                         ("portfolio_n300", 2.0), ("trajectory_N2000", 2.0),
                                         ("portfolio_n2000", 1.0), ("portfolio_n2500", 1.0)])
def test_refined_solve_matches_oracle(name, spread):
    makers = dict(SMALL, trajectory_N2000=lambda: trajectory_socp(N=2000, seed=5),
                  portfolio_n2000=lambda: portfolio_socp(n=2000, k=60, seed=6),
                  # budget and risk-cone rows of 2500 entries: the row kernels' long-row blocks
                  portfolio_n2500=lambda: portfolio_socp(n=2500, k=30, seed=7))
    prob = makers[name]()
    s, z, _, _ = random_cone_iterate(prob.l, prob.q, seed=6, scale_spread=spread)
    S = _setup(prob)
    S.kkt_factor_at(T(s), T(z))
    rng = np.random.default_rng(1)
    r = rng.standard_normal(S.N)
    import torch
    x = torch.zeros(S.N, dtype=torch.float64, device="cuda")
    steps, berr = S.kkt_solve(T(r), x)
    x = N(x)
    K = _oracle_K(prob, s, z)
    # backward error recomputed on the CPU (normwise, against the unregularised K)
    normK = float(abs(K).sum(axis=1).max())
    be = np.max(np.abs(K @ x - r)) / (normK * np.max(np.abs(x)) + np.max(np.abs(r)))
    assert be <= 1e-10 and berr <= 1e-10
    ks = ok.KKTSolver(K, ok.reg_signs(prob), 1e-8, max_refine=10, tol=1e-14)
    xo = ks.solve(r)
    if S.N <= 4000:
        # forward error bounded by the condition number times the backward errors
        cond = np.linalg.cond(K.toarray(), p=np.inf)
        tol = max(1e-9, 10.0 * cond * max(be, 1e-16))
        assert rel_inf(x, xo, floor=0.0) <= tol, (rel_inf(x, xo, floor=0.0), tol, cond)


@pytest.mark.parametrize("name", ["dense_qp_c1", "trajectory_N12", "portfolio_n300"])
def test_pivot_reciprocals_within_two_ulp(name):
    """The factor stores 1/d_j computed by Newton–Raphson from the hardware's approximate
    reciprocal; it must agree with the correctly rounded quotient to ≤ 2 ulp."""
    prob = SMALL[name]()
    s, z, _, _ = random_cone_iterate(prob.l, prob.q, seed=8, scale_spread=3.0)
    S = _setup(prob)
    S.kkt_factor_at(T(s), T(z))
    _, _, D = S.factor_dense()
    dinv = S.pivot_reciprocals()
    exact = 1.0 / D
    ulp = np.spacing(np.abs(exact))
    assert np.all(np.abs(dinv - exact) <= 2 * ulp)


def test_dataflow_wait_times_out_into_an_error_status():
    """The dataflow kernels' dependency wait never waits without bound: a probe waiting
    on a flag that nothing publishes gives up after a short poll budget and reports
    DEVICE_TIMEOUT; the context stays usable afterwards."""
    import torch
    import paper_2603_29197_gb300 as q
    from paper_2603_29197_gb300 import _lib
    lib = q.load()
    assert lib.qoco_gpu_selftest_wait_timeout(0, None) == _lib.ERR_INVALID_ARG
    rc = lib.qoco_gpu_selftest_wait_timeout(200000, None)
    assert rc == _lib.ERR_DEVICE_TIMEOUT
    # the device still works
    a = torch.ones(4, dtype=torch.float64, device="cuda")
    assert float((a * 2).sum().item()) == 8.0


def test_solve_with_a_one_poll_wait_budget_stops_with_device_timeout():
    """settings.wait_polls bounds every dependency wait of the real dataflow factor and
    solve kernels: with a budget of one poll, a front whose children are still being
    factored gives up at once, every block leaves, and qoco_gpu_solve returns
    DEVICE_TIMEOUT instead of hanging.  A solver with the default budget then solves the
    same problem in the same context."""
    import paper_2603_29197_gb300 as q
    from paper_2603_29197_gb300 import _lib
    from workloads import trajectory_socp
    prob = trajectory_socp(N=2000, seed=11)
    S = q.Solver(prob, wait_polls=1)
    assert S.solve() == _lib.ERR_DEVICE_TIMEOUT
    S.close()
    S = q.Solver(prob)
    assert S.solve() == 0
    assert_certificate(prob, S.solution())
    S.close()
