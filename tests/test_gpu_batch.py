"""Batched solves (qoco_gpu_setup_batch): many independent instances in one
interior-point loop with per-instance scalars, through the C ABI.

* A heterogeneous small batch (MPC instances of different horizons, a dense QP, a
  portfolio SOCP, a trajectory SOCP) matches the oracle instance by instance: objective
  1e-6, x, y, z 1e-5 relative, status solved, and the iteration at which each instance
  met the stopping test within 3 of the oracle's count.
* Each instance of a batch follows the single-problem path: same iteration count and
  the same solution to rounding as a stand-alone solve.
* The MPC batch of 4096 instances (horizons U{10..60}, state 4, control 2, Q³ input cone,
  box bounds) solves every instance; a seeded sample of 24 instances matches the oracle.
"""
import numpy as np
import pytest

from oracle import ipm
from workloads import dense_qp, mpc_batch, portfolio_socp, trajectory_socp
from _gpu_util import assert_certificate, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_2603_29197_gb300 as qq
    return qq


def _mixed_batch():
    probs = mpc_batch(count=8, tmin=10, tmax=30, seed=3)
    probs += [dense_qp(n=60, p=10, m=90, rank=8, density=0.1, seed=4), portfolio_socp(n=80, k=8, seed=5),
              trajectory_socp(N=40, seed=6)]
    probs += mpc_batch(count=3, tmin=40, tmax=60, seed=7)
    return probs


def _check_instance(prob, sol, ref):
    pobj = 0.5 * sol["x"] @ (prob.P @ sol["x"] + prob.P.T @ sol["x"] - prob.P.diagonal() * sol["x"]) \
        + prob.c @ sol["x"]
    assert abs(pobj - ref.pobj) <= 1e-6 * max(1.0, abs(ref.pobj)), (pobj, ref.pobj)
    assert rel_inf(sol["x"], ref.x) <= 1e-5
    if prob.p:
        assert rel_inf(sol["y"], ref.y) <= 1e-5
    assert rel_inf(sol["z"], ref.z) <= 1e-5
    assert_certificate(prob, sol)


def test_heterogeneous_batch_matches_oracle(q):
    probs = _mixed_batch()
    S = q.BatchSolver(probs)
    assert q.load().qoco_gpu_batch_size(S._h) == len(probs)
    assert S.solve() == 0
    info = S.batch_info()
    sols = S.instance_solutions()
    for i, prob in enumerate(probs):
        ref = ipm.solve(prob)
        assert ref.status == "solved"
        assert info["status"][i] == 0
        assert abs(int(info["iters"][i]) - ref.iters) <= 3, (i, info["iters"][i], ref.iters)
        assert abs(info["pobj"][i] - ref.pobj) <= 1e-6 * max(1.0, abs(ref.pobj))
        _check_instance(prob, sols[i], ref)
    S.close()


def test_batch_instances_follow_the_single_problem_path(q):
    probs = mpc_batch(count=5, tmin=10, tmax=60, seed=11)
    S = q.BatchSolver(probs)
    assert S.solve() == 0
    info = S.batch_info()
    sols = S.instance_solutions()
    for i, prob in enumerate(probs):
        one = q.Solver(prob)
        assert one.solve() == 0
        ref = one.solution()
        assert int(info["iters"][i]) == ref["info"]["iters"]
        for k in ("x", "z", "s"):
            assert rel_inf(sols[i][k], ref[k]) <= 1e-8, (i, k)
        one.close()
    S.close()


def test_mpc_batch_4096(q):
    probs = mpc_batch(count=4096, seed=0)
    S = q.BatchSolver(probs)
    assert S.solve() == 0
    info = S.batch_info()
    assert np.all(info["status"] == 0)
    sols = S.instance_solutions()
    rng = np.random.default_rng(0)
    for i in sorted(rng.choice(len(probs), size=24, replace=False)):
        ref = ipm.solve(probs[i])
        assert ref.status == "solved"
        _check_instance(probs[i], sols[i], ref)
    S.close()
