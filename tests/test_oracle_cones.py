"""Pins for oracle/cones.py: identities of the SOC Jordan algebra and of the
Nesterov–Todd scaling, brute force for the max step, Moreau decomposition for the
projection.  None of these retypes the oracle's formulas."""
import math

import numpy as np
import pytest

from oracle import cones
from workloads import random_cone_iterate

LAYOUTS = [(0, [2]), (0, [3]), (5, [4]), (3, [2, 3, 4, 7]), (0, [201]), (7, []), (4, [4] * 6 + [33])]


def _J(d):
    J = -np.eye(d)
    J[0, 0] = 1.0
    return J


@pytest.mark.parametrize("l,q", LAYOUTS)
@pytest.mark.parametrize("spread", [0.0, 3.0])
def test_nt_scaling_identities(l, q, spread):
    s, z, _, _ = random_cone_iterate(l, q, seed=11 + l + len(q), scale_spread=spread)
    W = cones.NTScaling(s, z, l, q)
    # Wz = W^{-1}s = λ
    lam_z = W.apply_W(z)
    lam_s = W.apply_Winv(s)
    np.testing.assert_allclose(lam_z, lam_s, rtol=1e-10, atol=1e-12 * np.abs(lam_z).max())
    np.testing.assert_allclose(W.lam, lam_z, rtol=1e-14, atol=0)
    # sᵀz = λᵀλ
    assert math.isclose(float(s @ z), float(W.lam @ W.lam), rel_tol=1e-10)
    # W² z = s  (the scaling maps z to s)
    np.testing.assert_allclose(W.apply_W(W.apply_W(z)), s, rtol=1e-9, atol=1e-12 * np.abs(s).max())
    for k, (o, d) in enumerate(cones.blocks(l, q)):
        Wk = W.W_block(k)
        # closed form of the square, W W⁻¹ = I, symmetry, w̄ᵀJw̄ = 1
        np.testing.assert_allclose(Wk @ Wk, W.W2_block(k), rtol=1e-10,
                                   atol=1e-12 * np.abs(Wk).max() ** 2)
        np.testing.assert_allclose(Wk @ W.Winv_block(k), np.eye(d), atol=1e-9)
        np.testing.assert_allclose(Wk, Wk.T, atol=0)
        wb = W.wbar[k]
        assert math.isclose(float(wb @ _J(d) @ wb), 1.0, rel_tol=1e-12)
        # λ is in the interior of the cone
        assert W.lam[o] > np.linalg.norm(W.lam[o + 1:o + d])
    if l:
        assert np.all(W.lam[:l] > 0)
        np.testing.assert_allclose(W.W2_orthant(), s[:l] / z[:l], rtol=1e-14)


def _spectral(u):
    """Eigenvalues u0 ± ‖u1‖ and the Jordan frame of one SOC element."""
    u1 = u[1:]
    t = np.linalg.norm(u1)
    dirn = u1 / t if t > 0 else np.eye(u1.size)[0]
    c1 = 0.5 * np.concatenate([[1.0], dirn])
    c2 = 0.5 * np.concatenate([[1.0], -dirn])
    return u[0] + t, u[0] - t, c1, c2


@pytest.mark.parametrize("l,q", LAYOUTS)
def test_jordan_identities(l, q):
    rng = np.random.default_rng(5)
    m = l + sum(q)
    u, v = rng.standard_normal(m), rng.standard_normal(m)
    e = cones.identity(l, q)
    np.testing.assert_allclose(cones.jordan_product(e, u, l, q), u, atol=1e-15)
    np.testing.assert_allclose(cones.jordan_product(u, v, l, q),
                               cones.jordan_product(v, u, l, q), atol=1e-14)
    # u∘u through the spectral decomposition: (λ1 c1 + λ2 c2)² = λ1² c1 + λ2² c2
    uu = cones.jordan_product(u, u, l, q)
    np.testing.assert_allclose(uu[:l], u[:l] ** 2)
    for o, d in cones.blocks(l, q):
        a1, a2, c1, c2 = _spectral(u[o:o + d])
        np.testing.assert_allclose(uu[o:o + d], a1 * a1 * c1 + a2 * a2 * c2, rtol=1e-12, atol=1e-12)
    # division inverts the product for λ in the interior
    s, z, _, _ = random_cone_iterate(l, q, seed=3)
    lam = cones.NTScaling(s, z, l, q).lam
    w = cones.jordan_division(lam, v, l, q)
    np.testing.assert_allclose(cones.jordan_product(lam, w, l, q), v, rtol=1e-10, atol=1e-10)
    # λ\(λ∘λ) = λ
    np.testing.assert_allclose(
        cones.jordan_division(lam, cones.jordan_product(lam, lam, l, q), l, q), lam,
        rtol=1e-10, atol=1e-12)


def _bisect_step(u, du, l, q, hi=1e6, iters=200):
    if cones.in_cone(u + hi * du, l, q):
        return math.inf
    lo = 0.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if cones.in_cone(u + mid * du, l, q):
            lo = mid
        else:
            hi = mid
    return lo


@pytest.mark.parametrize("l,q", LAYOUTS)
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_max_step_matches_bisection(l, q, seed):
    s, _, ds, _ = random_cone_iterate(l, q, seed=seed)
    a = cones.max_step(s, ds, l, q)
    b = _bisect_step(s, ds, l, q)
    if math.isinf(b):
        assert math.isinf(a) or a > 1e5
    else:
        assert math.isclose(a, b, rel_tol=1e-9), (a, b)


def test_max_step_special_cases():
    # direction inside the cone: unbounded step
    u = np.array([2.0, 0.5, -0.3])
    assert math.isinf(cones.max_step(u, np.array([1.0, 0.1, 0.2]), 0, [3]))
    # pure shrink towards the origin: step until u + α du = 0 on the axis
    assert math.isclose(cones.max_step(np.array([1.0, 0.0]), np.array([-1.0, 0.0]), 0, [2]), 1.0)
    # orthant: min ratio
    assert math.isclose(cones.max_step(np.array([1.0, 2.0]), np.array([-0.5, -4.0]), 2, []), 0.5)
    # boundary direction (a = 0): linear case
    u = np.array([1.0, 0.0])
    du = np.array([0.0, 1.0])
    assert math.isclose(cones.max_step(u, du, 0, [2]), _bisect_step(u, du, 0, [2]), rel_tol=1e-9)


@pytest.mark.parametrize("l,q", LAYOUTS)
def test_projection_moreau(l, q):
    rng = np.random.default_rng(9)
    m = l + sum(q)
    for _ in range(5):
        v = 3.0 * rng.standard_normal(m)
        pv = cones.project(v, l, q)
        pm = cones.project(-v, l, q)
        # v = Π(v) − Π(−v), both in K, Π(v) ⊥ Π(−v) (K self-dual)
        np.testing.assert_allclose(pv - pm, v, atol=1e-12)
        assert cones.in_cone(pv, l, q, tol=1e-12) and cones.in_cone(pm, l, q, tol=1e-12)
        assert abs(float(pv @ pm)) < 1e-10 * (1.0 + float(v @ v))


def test_projection_brute_force_small():
    from scipy.optimize import minimize
    v = np.array([0.3, 1.2, -0.7])
    cons = {"type": "ineq", "fun": lambda x: x[0] - np.linalg.norm(x[1:])}
    res = minimize(lambda x: 0.5 * np.sum((x - v) ** 2), np.array([2.0, 0.0, 0.0]),
                   constraints=[cons], method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
    np.testing.assert_allclose(cones.project(v, 0, [3]), res.x, atol=1e-6)


@pytest.mark.parametrize("l,q", LAYOUTS)
def test_shift_into_cone(l, q):
    rng = np.random.default_rng(4)
    m = l + sum(q)
    u = rng.standard_normal(m)
    su = cones.shift_into_cone(u, l, q)
    # the smallest eigenvalue over all cones becomes exactly 1 (when a shift happens)
    eig = list(su[:l])
    for o, d in cones.blocks(l, q):
        eig.append(su[o] - np.linalg.norm(su[o + 1:o + d]))
    assert math.isclose(min(eig), 1.0, rel_tol=1e-12)
    # an interior point is left alone
    s, _, _, _ = random_cone_iterate(l, q, seed=1)
    np.testing.assert_array_equal(cones.shift_into_cone(s, l, q), s)
