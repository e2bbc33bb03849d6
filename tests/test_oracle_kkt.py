"""Pins for oracle/kkt.py: the assembled KKT blocks against a dense construction
from the problem data, the refined solve against a dense solve, and the textbook
LDLᵀ against reconstruction and against Cholesky."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import cones, kkt
from workloads import dense_qp, portfolio_socp, random_cone_iterate, trajectory_socp


def _small_problems():
    return [dense_qp(n=30, p=5, m=40, rank=4, density=0.2, seed=1),
            trajectory_socp(N=12, seed=2),
            portfolio_socp(n=25, k=4, seed=3)]


@pytest.mark.parametrize("prob", _small_problems(), ids=lambda p: p.name)
def test_assemble_blocks(prob):
    s, z, _, _ = random_cone_iterate(prob.l, prob.q, seed=7)
    W = cones.NTScaling(s, z, prob.l, prob.q)
    K = kkt.assemble(prob, kkt.z_block(W, prob.m)).toarray()
    n, p, m = prob.n, prob.p, prob.m
    Pu = prob.P.toarray()
    Pf = np.triu(Pu) + np.triu(Pu, 1).T
    np.testing.assert_array_equal(K[:n, :n], Pf)
    np.testing.assert_array_equal(K[n:n + p, :n], prob.A.toarray())
    np.testing.assert_array_equal(K[n + p:, :n], prob.G.toarray())
    np.testing.assert_array_equal(K, K.T)
    assert not K[n:n + p, n:].any()
    # z block: −W² built blockwise, W² z = s (so −K_zz z = s)
    np.testing.assert_allclose(-K[n + p:, n + p:] @ z, s, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("prob", _small_problems(), ids=lambda p: p.name)
def test_refined_solve_matches_dense(prob):
    s, z, _, _ = random_cone_iterate(prob.l, prob.q, seed=8)
    W = cones.NTScaling(s, z, prob.l, prob.q)
    K = kkt.assemble(prob, kkt.z_block(W, prob.m))
    ks = kkt.KKTSolver(K, kkt.reg_signs(prob), 1e-8, max_refine=10, tol=1e-14)
    r = np.random.default_rng(0).standard_normal(K.shape[0])
    x = ks.solve(r)
    xd = np.linalg.solve(K.toarray(), r)
    np.testing.assert_allclose(x, xd, rtol=1e-7, atol=1e-9 * np.abs(xd).max())
    assert ks.backward_error(x, r) <= 1e-13


def test_dense_ldlt_reconstruction_and_cholesky():
    rng = np.random.default_rng(1)
    B = rng.standard_normal((9, 9))
    S = B @ B.T + 9 * np.eye(9)
    L, d = kkt.dense_ldlt(S)
    np.testing.assert_allclose(L @ np.diag(d) @ L.T, S, atol=1e-12)
    C = sla.cholesky(S, lower=True)
    np.testing.assert_allclose(d, np.diag(C) ** 2, rtol=1e-12)
    np.testing.assert_allclose(L, C / np.diag(C), atol=1e-12)
    # quasidefinite with signs: pivots carry the block signs
    prob = dense_qp(n=12, p=3, m=10, rank=3, density=0.3, seed=2)
    K = kkt.assemble(prob, kkt.initial_W2(prob)).toarray()
    sg = kkt.reg_signs(prob)
    Ke = K + 1e-8 * np.diag(sg)
    L, d = kkt.dense_ldlt(Ke, signs=sg)
    np.testing.assert_allclose(L @ np.diag(d) @ L.T, Ke, atol=1e-9)
    assert np.all(np.sign(d) == sg)


def test_dense_ldlt_dynamic_regularisation():
    # a zero pivot in the natural order is replaced by sign·1e-7
    M = np.array([[0.0, 1.0], [1.0, 0.0]])
    L, d = kkt.dense_ldlt(M, signs=np.array([1.0, -1.0]))
    assert d[0] == 1e-7
    assert np.isclose(d[1], -1.0 / 1e-7)
