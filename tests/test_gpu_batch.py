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


@pytest.mark.parametrize("schedule", [1, 2, 3, 4, 5])
def test_batch_schedules_match_the_oracle(q, schedule):
    """Every layout of the per-instance factor/solve kernels (4 or 8 warps per CTA,
    tiny fronts one per thread or every front one warp) and the shared kernels solve the
    same instances to the oracle's tolerances."""
    probs = mpc_batch(count=48, tmin=10, tmax=60, seed=21)
    S = q.BatchSolver(probs, batch_schedule=schedule)
    assert S.solve() == 0
    assert S.info()["batch_schedule_used"] == schedule
    info = S.batch_info()
    assert np.all(info["status"] == 0)
    sols = S.instance_solutions()
    for i in (0, 7, 19, 33, 47):
        ref = ipm.solve(probs[i])
        assert ref.status == "solved"
        assert abs(int(info["iters"][i]) - ref.iters) <= 3
        _check_instance(probs[i], sols[i], ref)
    S.close()


def test_batch_schedule_autotune_picks_a_candidate(q):
    probs = mpc_batch(count=32, tmin=10, tmax=60, seed=22)
    S = q.BatchSolver(probs)
    assert S.info()["batch_schedule_used"] == 0  # chosen on the first factorisation
    assert S.solve() == 0
    used = S.info()["batch_schedule_used"]
    assert used in (1, 2, 3, 4, 5)
    sols = S.instance_solutions()
    T = q.BatchSolver(probs, batch_schedule=used)
    assert T.solve() == 0
    for a, b in zip(sols, T.instance_solutions()):
        for k in ("x", "y", "z", "s"):
            assert np.array_equal(a[k], b[k])  # the tuned run is the fixed candidate's run
    S.close()
    T.close()


def test_batch_with_a_front_beyond_one_warp_uses_the_shared_kernels(q):
    probs = mpc_batch(count=4, tmin=10, tmax=20, seed=23) + [dense_qp(n=60, p=10, m=90, rank=8, density=0.1, seed=4)]
    S = q.BatchSolver(probs)
    assert S.info()["max_front"] > 48
    assert S.info()["batch_schedule_used"] == 5
    assert S.solve() == 0
    S.close()
