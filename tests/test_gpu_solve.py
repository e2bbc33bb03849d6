"""Whole interior-point solves on the GPU (qoco_gpu_setup → qoco_gpu_solve →
qoco_gpu_get_solution) against the oracle on the same seeded instances: objective
within 1e-6 relative, x, y, z within 1e-5 (‖Δ‖∞ / max(1, ‖v‖∞)), plus an
independent KKT certificate of the returned point."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ipm
from workloads import (Problem, dense_qp, lasso_qp, mpc_batch, portfolio_socp,
                       trajectory_socp)

from _gpu_util import assert_certificate, rel_inf

pytestmark = pytest.mark.gpu


def _lp(n=4, seed=0):
    rng = np.random.default_rng(seed)
    G = np.vstack([np.eye(n), -np.eye(n), rng.standard_normal((2 * n, n))])
    h = np.concatenate([np.ones(2 * n), rng.uniform(0.2, 1.0, 2 * n)])
    return Problem(n=n, m=G.shape[0], p=0, P=sp.csc_matrix((n, n)), c=rng.standard_normal(n),
                   A=sp.csc_matrix((0, n)), b=np.zeros(0), G=sp.csc_matrix(G), h=h,
                   l=G.shape[0], q=[], name=f"lp_n{n}")


def _soc_projection(v):
    q = len(v)
    return Problem(n=q, m=q, p=0, P=sp.identity(q, format="csc"), c=-np.asarray(v, float),
                   A=sp.csc_matrix((0, q)), b=np.zeros(0), G=-sp.identity(q, format="csc"),
                   h=np.zeros(q), l=0, q=[q], name=f"soc_proj_q{q}")


def _eq_qp(seed=0):
    rng = np.random.default_rng(seed)
    n, p = 40, 10
    B = rng.standard_normal((n, n))
    P = B @ B.T + np.eye(n)
    A = rng.standard_normal((p, n))
    return Problem(n=n, m=0, p=p, P=sp.csc_matrix(np.triu(P)), c=rng.standard_normal(n),
                   A=sp.csc_matrix(A), b=rng.standard_normal(p), G=sp.csc_matrix((0, n)),
                   h=np.zeros(0), l=0, q=[], name="equality_qp")


CASES = {
    "dense_qp_c1": lambda: dense_qp(),
    "dense_qp_small": lambda: dense_qp(n=60, p=10, m=90, rank=8, density=0.1, seed=4),
    "trajectory_N200": lambda: trajectory_socp(N=200, seed=0),
    "trajectory_N1000": lambda: trajectory_socp(N=1000, seed=3),
    "portfolio_n200": lambda: portfolio_socp(n=200, k=20, seed=0),
    "portfolio_n1500": lambda: portfolio_socp(n=1500, k=60, seed=1),
    "lasso_small": lambda: lasso_qp(rows=300, cols=600, density=0.02, seed=4),
    "mpc_T": lambda: mpc_batch(count=3, seed=5)[2],
    "lp_n4": lambda: _lp(4, 1),
    "soc_projection": lambda: _soc_projection([0.1, 0.0, 5.0, -1.0, 2.0]),
    "equality_qp": lambda: _eq_qp(),
}


@pytest.fixture(scope="module")
def q():
    import paper_2603_29197_gb300 as qq
    return qq


@pytest.mark.parametrize("name", list(CASES))
def test_solve_matches_oracle(q, name):
    prob = CASES[name]()
    ref = ipm.solve(prob)
    assert ref.status == "solved"
    S = q.Solver(prob)
    status = S.solve()
    sol = S.solution()
    info = sol["info"]
    assert status == 0, info
    assert abs(info["pobj"] - ref.pobj) <= 1e-6 * max(1.0, abs(ref.pobj)), (info["pobj"], ref.pobj)
    assert rel_inf(sol["x"], ref.x) <= 1e-5
    assert rel_inf(sol["y"], ref.y) <= 1e-5
    assert rel_inf(sol["z"], ref.z) <= 1e-5
    assert abs(info["iters"] - ref.iters) <= 3, (info["iters"], ref.iters)
    assert_certificate(prob, sol)
    assert info["kernel_launches"] > 0


def test_repeated_solves_are_identical(q):
    prob = trajectory_socp(N=300, seed=2)
    S = q.Solver(prob)
    assert S.solve() == 0
    a = S.solution()
    assert S.solve() == 0
    b = S.solution()
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["z"], b["z"])
    assert a["info"]["iters"] == b["info"]["iters"]


def test_profiling_modes(q):
    """Mode 1 times every phase, mode 2 the factorisation alone (what bench.py uses inside
    its timed region), 0 turns it off; the solution does not depend on the mode."""
    prob = trajectory_socp(N=300, seed=2)
    S = q.Solver(prob)
    S.set_profiling(True)
    assert S.solve() == 0
    full = S.profile()
    x1 = S.solution()["x"]
    S.set_profiling(2)
    assert S.solve() == 0
    fac = S.profile()
    x2 = S.solution()["x"]
    S.set_profiling(False)
    iters = S.info()["iters"]
    assert full["factor"]["calls"] == iters + 1 and full["solve"]["calls"] >= 2 * iters
    assert full["cone"]["calls"] > 0 and full["row"]["calls"] > 0
    assert fac["factor"]["calls"] == iters + 1 and fac["factor"]["ms"] > 0.0
    assert fac["solve"]["calls"] == fac["cone"]["calls"] == fac["row"]["calls"] == 0
    np.testing.assert_array_equal(x1, x2)
    assert S.lib.qoco_gpu_set_profiling(S._h, 3) == -10  # QOCO_GPU_ERR_INVALID_ARG
    S.close()


def test_max_iter_status(q):
    prob = dense_qp(n=60, p=10, m=90, rank=8, density=0.1, seed=4)
    S = q.Solver(prob, max_iter=2)
    assert S.solve() in (1, 2)
    assert S.info()["iters"] == 2


def test_orderings_agree(q):
    prob = trajectory_socp(N=150, seed=6)
    sols = []
    for order in (q.ORDER_AMD, q.ORDER_ND, q.ORDER_NATURAL):
        S = q.Solver(prob, ordering=order)
        assert S.solve() == 0
        sols.append(S.solution())
    for s in sols[1:]:
        assert rel_inf(s["x"], sols[0]["x"]) <= 1e-6
        assert abs(s["info"]["pobj"] - sols[0]["info"]["pobj"]) <= 1e-7 * abs(sols[0]["info"]["pobj"])


def test_one_variable_problem(q):
    # min x² + x  s.t.  x ≥ 0  (G = −1, h = 0): the bound is active, x = 0
    prob = Problem(n=1, m=1, p=0, P=sp.csc_matrix([[2.0]]), c=np.array([1.0]), A=sp.csc_matrix((0, 1)),
                   b=np.zeros(0), G=sp.csc_matrix([[-1.0]]), h=np.zeros(1), l=1, q=[], name="one_var")
    ref = ipm.solve(prob)
    S = q.Solver(prob)
    assert S.solve() == 0
    sol = S.solution()
    assert abs(sol["x"][0] - ref.x[0]) <= 1e-6 and abs(sol["x"][0]) <= 1e-6
    assert abs(sol["z"][0] - 1.0) <= 1e-5  # the multiplier equals the gradient at 0
    S.close()


def test_infeasible_problem_is_not_reported_solved(q):
    # x ≥ 1 and x ≤ −1: no feasible point; the loop must stop at max_iter (or on a
    # numerical failure) without claiming a solution
    prob = Problem(n=1, m=2, p=0, P=sp.csc_matrix((1, 1)), c=np.array([1.0]), A=sp.csc_matrix((0, 1)),
                   b=np.zeros(0), G=sp.csc_matrix([[-1.0], [1.0]]), h=np.array([-1.0, -1.0]), l=2, q=[],
                   name="infeasible")
    S = q.Solver(prob, max_iter=40)
    status = S.solve()
    assert status in (2, -5), status  # MAX_ITER or ERR_NUMERICAL
    S.close()
