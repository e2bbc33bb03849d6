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
* A batch's analysis orders each distinct instance pattern once: its factor flops, L
  entries and supernodes are the sums of the instances' own analyses (host-only, the
  same ordering), with patterns repeated and mixed, and its solves match the oracle.
* The persistent batched kernel (one launch per batched solve, the default when every
  front fits one warp) and each of its tile configurations (tuned, or fixed by schedules
  7–12) match the oracle instance by
  instance, are bitwise reproducible, and agree with the level-loop schedules.
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


@pytest.mark.parametrize("ordering", [1, 2])
def test_batch_analysis_is_the_sum_of_the_instances(q, ordering):
    # horizons 10..13 repeat the same four MPC patterns; a dense QP and a portfolio SOCP
    # sit between them
    probs = mpc_batch(count=12, tmin=10, tmax=13, seed=21)
    probs = probs[:6] + [dense_qp(n=40, p=8, m=60, rank=6, density=0.1, seed=22),
                         portfolio_socp(n=50, k=6, seed=23)] + probs[6:]
    S = q.BatchSolver(probs, ordering=ordering)
    info = S.info()
    assert info["ordering_used"] == ordering
    one = [q.analyze(pr, ordering=ordering)[0] for pr in probs]
    assert info["factor_flops"] == sum(o["factor_flops"] for o in one)
    assert info["l_nnz"] == sum(o["l_nnz"] for o in one)
    assert info["n_supernodes"] == sum(o["n_supernodes"] for o in one)
    assert S.solve() == 0
    bi = S.batch_info()
    sols = S.instance_solutions()
    for i in (0, 6, 7, len(probs) - 1):
        ref = ipm.solve(probs[i])
        assert bi["status"][i] == 0
        _check_instance(probs[i], sols[i], ref)
    S.close()


@pytest.mark.parametrize("schedule", [1, 2, 3, 4, 5, 6])
def test_batch_schedules_match_the_oracle(q, schedule):
    """Every layout of the per-instance factor/solve kernels (4 or 8 warps per CTA,
    tiny fronts one per thread or every front one warp), the shared kernels and the
    persistent batched kernel solve the same instances to the oracle's tolerances."""
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


@pytest.mark.parametrize("schedule", [7, 8, 9, 10, 11, 12])
def test_persistent_kernel_fixed_tiles_match_the_oracle(q, schedule):
    """Every tile of the persistent kernel (1, 2 or 4 warps per CTA; 16 or 32 resident
    warps per SM), fixed instead of tuned, solves the same instances to the oracle's
    tolerances; the tuning times only some of them."""
    probs = mpc_batch(count=48, tmin=10, tmax=60, seed=21)
    S = q.BatchSolver(probs, batch_schedule=schedule)
    assert S.solve() == 0
    info = S.info()
    assert info["batch_schedule_used"] == 6
    assert info["batch_warps"] == 1 << ((schedule - 7) // 2)
    assert info["batch_warps_per_sm"] == (32 if (schedule - 7) % 2 else 16)
    bi = S.batch_info()
    assert np.all(bi["status"] == 0)
    sols = S.instance_solutions()
    for i in (0, 19, 47):
        ref = ipm.solve(probs[i])
        assert abs(int(bi["iters"][i]) - ref.iters) <= 3
        _check_instance(probs[i], sols[i], ref)
    S.close()


def test_persistent_batched_kernel_is_the_default_and_reproducible(q):
    """Batches whose fronts all fit one warp are solved by the persistent kernel (one
    launch per batched solve, its tile configuration autotuned at the first solve):
    repeated solves are bitwise equal, and every instance agrees with the level-loop
    shared kernels (schedule 5) to 1e-8 with the same iteration count up to one."""
    probs = mpc_batch(count=96, tmin=10, tmax=60, seed=22)
    S = q.BatchSolver(probs)
    assert S.info()["batch_schedule_used"] == 6
    assert S.solve() == 0
    first = [dict((k, v.copy()) for k, v in d.items()) for d in S.instance_solutions()]
    assert S.solve() == 0
    assert S.info()["kernel_launches"] <= 3  # the batched kernel, the summary (one graph)
    for a, b in zip(first, S.instance_solutions()):
        for k in ("x", "y", "z", "s"):
            assert np.array_equal(a[k], b[k])
    fi = S.batch_info()
    T = q.BatchSolver(probs, batch_schedule=5)
    assert T.solve() == 0
    ti = T.batch_info()
    for i, (a, b) in enumerate(zip(first, T.instance_solutions())):
        assert abs(int(fi["iters"][i]) - int(ti["iters"][i])) <= 1, i
        for k in ("x", "y", "z"):
            assert rel_inf(a[k], b[k]) <= 1e-8, (i, k)
    S.close()
    T.close()


@pytest.mark.parametrize("wait_polls", [1])
def test_persistent_batched_kernel_needs_no_device_waits(q, wait_polls):
    """The persistent kernel's CTAs never wait on one another (each owns whole
    instances), so even a one-poll wait budget leaves its solves unaffected."""
    probs = mpc_batch(count=40, tmin=10, tmax=60, seed=24)
    S = q.BatchSolver(probs, wait_polls=wait_polls)
    assert S.solve() == 0
    assert np.all(S.batch_info()["status"] == 0)
    S.close()


def test_batch_with_a_front_beyond_one_warp_uses_the_shared_kernels(q):
    probs = mpc_batch(count=4, tmin=10, tmax=20, seed=23) + [dense_qp(n=60, p=10, m=90, rank=8, density=0.1, seed=4)]
    S = q.BatchSolver(probs)
    assert S.info()["max_front"] > 48
    assert S.info()["batch_schedule_used"] == 5
    assert S.solve() == 0
    S.close()


def test_persistent_batched_kernel_mixed_precision_matches_oracle(q):
    """Mixed precision on the persistent batched kernel: every front factored in FP32,
    the solves and refinement in FP64 (an instance whose refinement misses the target on
    an FP32 factor is refactored in FP64); every instance reaches the oracle's solution
    to the plain form's tolerances."""
    probs = mpc_batch(count=64, tmin=10, tmax=60, seed=25)
    S = q.BatchSolver(probs, mixed_precision=1)
    assert S.info()["batch_schedule_used"] == 6
    assert S.solve() == 0
    info = S.batch_info()
    assert np.all(info["status"] == 0)
    sols = S.instance_solutions()
    for i in (0, 5, 17, 40, 63):
        ref = ipm.solve(probs[i])
        assert ref.status == "solved"
        assert abs(int(info["iters"][i]) - ref.iters) <= 3
        _check_instance(probs[i], sols[i], ref)
    S.close()
