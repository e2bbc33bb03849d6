"""Pins for oracle/ipm.py against closed forms and textbook special cases:
equality-constrained QP solved directly from its KKT system, vertex enumeration on
tiny LPs, projection onto one SOC, water-filling (portfolio with the risk cone
inactive), finite-horizon LQR by the Riccati recursion (MPC with inactive bounds),
the lasso subgradient certificate, and an independent KKT certificate at
termination."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cones, ipm
from workloads import (Problem, dense_qp, lasso_qp, mpc_instance, portfolio_socp,
                       trajectory_socp)


def _prob(P, c, A, b, G, h, l, q, name="t"):
    n = len(c)
    A = np.zeros((0, n)) if A is None else A
    return Problem(n=n, m=G.shape[0], p=A.shape[0], P=sp.csc_matrix(np.triu(P)), c=c,
                   A=sp.csc_matrix(A), b=np.asarray(b, float), G=sp.csc_matrix(G),
                   h=np.asarray(h, float), l=l, q=list(q), name=name)


def certificate(prob, r, tol=1e-6):
    """Independent optimality certificate from dense data."""
    Pu = prob.P.toarray()
    P = np.triu(Pu) + np.triu(Pu, 1).T
    A, G = prob.A.toarray(), prob.G.toarray()
    x, s, y, z = r.x, r.s, r.y, r.z
    rx = P @ x + prob.c + A.T @ y + G.T @ z
    ry = A @ x - prob.b
    rz = G @ x + s - prob.h
    scale = 1.0 + max(np.abs(prob.c).max(initial=0), np.abs(prob.b).max(initial=0),
                      np.abs(prob.h).max(initial=0))
    assert np.abs(rx).max(initial=0) <= tol * scale
    assert np.abs(ry).max(initial=0) <= tol * scale
    assert np.abs(rz).max(initial=0) <= tol * scale
    assert cones.in_cone(s, prob.l, prob.q, tol=1e-9) and cones.in_cone(z, prob.l, prob.q, tol=1e-9)
    pobj = 0.5 * x @ P @ x + prob.c @ x
    assert abs(s @ z) <= tol * (1.0 + abs(pobj))


def test_equality_qp_closed_form():
    rng = np.random.default_rng(0)
    n, p = 12, 4
    B = rng.standard_normal((n, n))
    P = B @ B.T + np.eye(n)
    c = rng.standard_normal(n)
    A = rng.standard_normal((p, n))
    b = rng.standard_normal(p)
    sol = np.linalg.solve(np.block([[P, A.T], [A, np.zeros((p, p))]]), np.concatenate([-c, b]))
    xe, ye = sol[:n], sol[n:]
    G = rng.standard_normal((6, n))
    h = G @ xe + 1e3  # inactive inequalities
    r = ipm.solve(_prob(P, c, A, b, G, h, 6, []))
    assert r.status == "solved"
    np.testing.assert_allclose(r.x, xe, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(r.y, ye, rtol=1e-5, atol=1e-5)
    assert np.abs(r.z).max() < 1e-6


def _vertex_lp(c, G, h):
    n = len(c)
    best, bestx, vals = np.inf, None, []
    for rows in itertools.combinations(range(G.shape[0]), n):
        Gs = G[list(rows)]
        if abs(np.linalg.det(Gs)) < 1e-10:
            continue
        x = np.linalg.solve(Gs, h[list(rows)])
        if np.all(G @ x <= h + 1e-9):
            f = float(c @ x)
            vals.append(f)
            if f < best:
                best, bestx = f, x
    vals = sorted(set(np.round(vals, 9)))
    unique = len(vals) < 2 or vals[1] - vals[0] > 1e-6
    return best, bestx, unique


@pytest.mark.parametrize("n,seed", [(2, 0), (2, 1), (3, 2), (3, 3), (4, 4), (4, 5)])
def test_tiny_lp_vertex_enumeration(n, seed):
    rng = np.random.default_rng(seed)
    k = 2 * n
    G = np.vstack([np.eye(n), -np.eye(n), rng.standard_normal((k, n))])
    h = np.concatenate([np.ones(2 * n), rng.uniform(0.2, 1.0, k)])
    c = rng.standard_normal(n)
    f, xv, unique = _vertex_lp(c, G, h)
    r = ipm.solve(_prob(np.zeros((n, n)), c, None, [], G, h, G.shape[0], []))
    assert r.status == "solved"
    assert abs(r.pobj - f) <= 1e-6 * max(1.0, abs(f))
    if unique:
        np.testing.assert_allclose(r.x, xv, atol=1e-5)


@pytest.mark.parametrize("v", [[0.3, 1.2, -0.7], [2.0, 0.3, 0.4], [-1.0, 0.2, 0.1, 0.3],
                               [0.1, 0.0, 5.0, -1.0, 2.0]])
def test_soc_projection_by_ipm(v):
    v = np.asarray(v, float)
    q = v.size
    r = ipm.solve(_prob(np.eye(q), -v, None, [], -np.eye(q), np.zeros(q), 0, [q]))
    assert r.status == "solved"
    np.testing.assert_allclose(r.x, cones.project(v, 0, [q]), atol=1e-6)


def _waterfill_exact(d, mu):
    """Exact solution of min Σ d_i x_i² − μᵀx, 1ᵀx = 1, x ≥ 0 by scanning the active set
    in decreasing μ (x_i = (μ_i − ν)/(2 d_i) on the active set)."""
    order = np.argsort(-mu)
    a = b = 0.0
    nu = None
    for j, i in enumerate(order):
        a += mu[i] / (2 * d[i])
        b += 1.0 / (2 * d[i])
        cand = (a - 1.0) / b
        nxt = mu[order[j + 1]] if j + 1 < len(order) else -np.inf
        if cand >= nxt and cand < mu[i]:
            nu = cand
            break
    return np.maximum(0.0, (mu - nu) / (2 * d))


def test_portfolio_waterfilling():
    prob = portfolio_socp(n=200, k=20, gamma_frac=1e3, seed=1)
    r = ipm.solve(prob)
    assert r.status == "solved"
    xw = _waterfill_exact(prob.meta["d"], prob.meta["mu"])
    np.testing.assert_allclose(r.x, xw, atol=1e-5)


def test_mpc_matches_lqr_riccati():
    rng = np.random.default_rng(3)
    nx, nu, T = 4, 2, 15
    Q, R_ = np.linalg.qr(rng.standard_normal((nx, nx)))
    A = Q @ np.diag(rng.uniform(0.8, 0.99, nx)) @ Q.T
    B = 0.5 * rng.standard_normal((nx, nu))
    x0 = rng.uniform(-1, 1, nx)
    prob = mpc_instance(T, A, B, x0, box=1e4, umax=1e4)
    r = ipm.solve(prob)
    assert r.status == "solved"
    # backward Riccati: stage cost ‖x‖² (k ≥ 1) + 0.1‖u‖², terminal ‖x_T‖²
    Rm = 0.1 * np.eye(nu)
    S = np.eye(nx)
    gains = []
    for k in range(T - 1, -1, -1):
        K = np.linalg.solve(Rm + B.T @ S @ B, B.T @ S @ A)
        gains.append(K)
        S = (np.eye(nx) if k >= 1 else 0 * np.eye(nx)) + A.T @ S @ (A - B @ K)
    gains = gains[::-1]
    x = x0.copy()
    xs, us = [], []
    for k in range(T):
        u = -gains[k] @ x
        x = A @ x + B @ u
        us.append(u)
        xs.append(x)
    ns = nx + nu
    for k in range(T):
        np.testing.assert_allclose(r.x[ns * k:ns * k + nu], us[k], atol=1e-5)
        np.testing.assert_allclose(r.x[ns * k + nu:ns * k + ns], xs[k], atol=1e-5)


def test_lasso_subgradient_certificate():
    prob = lasso_qp(rows=300, cols=600, density=0.02, seed=4)
    r = ipm.solve(prob, ipm.Settings(abstol=1e-9, reltol=1e-9))
    assert r.status == "solved"
    F, y, lam = prob.meta["F"], prob.meta["y"], prob.meta["lam"]
    cols = prob.meta["cols"]
    x = r.x[:cols]
    g = F.T @ (F @ x - y)
    assert np.abs(g).max() <= lam * (1 + 1e-6)
    supp = np.abs(x) > 1e-3 * np.abs(x).max()
    assert supp.any()
    np.testing.assert_allclose(g[supp], -lam * np.sign(x[supp]), rtol=1e-5)


@pytest.mark.parametrize("make", [lambda: dense_qp(), lambda: trajectory_socp(N=60, seed=1),
                                  lambda: portfolio_socp(n=150, k=10, seed=2)],
                         ids=["dense_qp", "trajectory_N60", "portfolio_n150"])
def test_kkt_certificate_at_termination(make):
    prob = make()
    r = ipm.solve(prob)
    assert r.status == "solved"
    certificate(prob, r)


@pytest.mark.parametrize("make", [
    lambda: dense_qp(n=40, p=10, m=60, rank=5, density=0.2, seed=3),
    lambda: trajectory_socp(N=30, seed=4),
    lambda: portfolio_socp(n=60, k=8, seed=5),
])
def test_directions_satisfy_the_linearised_newton_system(make):
    """Both search directions of an iteration (affine d_s = −λ∘λ and a combined one with
    the Mehrotra term and centring) solve the linearised optimality conditions at the
    current point, checked with the problem's dense matrices:
        PΔx + AᵀΔy + GᵀΔz = −r_x,  AΔx = −r_y,  GΔx + Δs = −r_z,  λ∘(WΔz + W⁻¹Δs) = d_s.
    A dropped or mis-signed term anywhere in the direction's right-hand side or in the
    Δs recovery breaks one of the four."""
    from oracle import kkt as kktmod
    from workloads import random_cone_iterate
    prob = make()
    rng = np.random.default_rng(7)
    n, p, m, l, q = prob.n, prob.p, prob.m, prob.l, prob.q
    x, y = rng.standard_normal(n), rng.standard_normal(p)
    s, z, _, _ = random_cone_iterate(l, q, seed=9)
    Pu = prob.P.toarray()
    P = np.triu(Pu) + np.triu(Pu, 1).T
    A, G = prob.A.toarray(), prob.G.toarray()
    rx = P @ x + prob.c + A.T @ y + G.T @ z
    ry = A @ x - prob.b
    rz = G @ x + s - prob.h
    W = cones.NTScaling(s, z, l, q)
    K = kktmod.assemble(prob, kktmod.z_block(W, m))
    ks = kktmod.KKTSolver(K, kktmod.reg_signs(prob), 1e-8, 10, 1e-12)
    lam = W.lam
    e = cones.identity(l, q)
    ds_aff = -cones.jordan_product(lam, lam, l, q)
    dx_a, dy_a, dz_a, dsa = ipm.newton_direction(prob, W, ks, rx, ry, rz, ds_aff)
    corr = cones.jordan_product(W.apply_Winv(dsa), W.apply_W(dz_a), l, q)
    ds_cmb = ds_aff - corr + 0.3 * float(s @ z) / cones.degree(l, q) * e
    for ds in (ds_aff, ds_cmb):
        dx, dy, dz, dsv = ipm.newton_direction(prob, W, ks, rx, ry, rz, ds)
        sc = 1.0 + max(np.abs(rx).max(), np.abs(rz).max(), np.abs(dx).max(), np.abs(dz).max())
        assert np.abs(P @ dx + A.T @ dy + G.T @ dz + rx).max() <= 1e-8 * sc
        if p:
            assert np.abs(A @ dx + ry).max() <= 1e-8 * sc
        assert np.abs(G @ dx + dsv + rz).max() <= 1e-8 * sc
        lhs = cones.jordan_product(lam, W.apply_W(dz) + W.apply_Winv(dsv), l, q)
        assert np.abs(lhs - ds).max() <= 1e-8 * (1.0 + np.abs(ds).max())
