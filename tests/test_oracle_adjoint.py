"""Pins of the oracle's adjoint (oracle/adjoint.py) against what the mathematics fixes:

* the complementarity block B = −Arw(z)⁻¹Arw(s) linearises the Jordan product:
  z ∘ (B dz) + s ∘ dz = 0 for every dz (checked with the oracle's Jordan product, an
  independent function pinned in test_oracle_cones.py);
* central finite differences of the oracle's solution map, run to tight tolerances, on
  an orthant-only QP (strictly complementary: agreement to ~1e-8) and on the portfolio
  SOCP with an active second-order cone (agreement limited to ~1e-3 by how close the
  final iterate sits to the cone's boundary);
* the closed form of an equality-constrained QP: with every inequality row inactive,
  v solves the reduced system [[P, Aᵀ], [A, 0]] v = (g_x, g_y), so ∂L/∂c = −v_x,
  ∂L/∂b = v_y and ∂L/∂h = 0.
"""
import copy

import numpy as np
import pytest

from oracle import adjoint, cones, ipm
from oracle import kkt as kktmod
from workloads import dense_qp, portfolio_socp, random_cone_iterate


@pytest.mark.parametrize("l,q", [(6, []), (0, [3]), (4, [2, 5, 3])])
def test_complementarity_block_linearises_the_jordan_product(l, q):
    s, z, _, _ = random_cone_iterate(l, q, seed=7)
    B = adjoint.complementarity_block(s, z, l, q).toarray()
    rng = np.random.default_rng(1)
    for _ in range(3):
        dz = rng.standard_normal(len(s))
        ds = B @ dz
        lin = cones.jordan_product(z, ds, l, q) + cones.jordan_product(s, dz, l, q)
        assert np.max(np.abs(lin)) <= 1e-12 * max(1.0, np.max(np.abs(s)) * np.max(np.abs(dz)))


def test_complementarity_block_is_minus_w2_on_the_orthant():
    s, z, _, _ = random_cone_iterate(9, [], seed=3)
    B = adjoint.complementarity_block(s, z, 9, []).toarray()
    W = cones.NTScaling(s, z, 9, [])
    assert np.allclose(np.diag(B), -W.W2_orthant(), rtol=1e-14, atol=0)


def _loss(prob, st, xref):
    r = ipm.solve(prob, st)
    assert r.status == "solved", r.status
    return float(np.sum((r.x - xref) ** 2)), r


def _fd_check(prob, tol, h_rel, rtol, groups):
    st = ipm.Settings(abstol=tol, reltol=tol, max_iter=100)
    xref = np.full(prob.n, 1.0 / prob.n)
    _, r = _loss(prob, st, xref)
    g = adjoint.backward(prob, r, 2.0 * (r.x - xref))
    rng = np.random.default_rng(0)
    for key, attr in groups:
        base = getattr(prob, attr)
        dense = isinstance(base, np.ndarray)
        vals = base if dense else base.data
        d = rng.standard_normal(vals.shape)
        h = h_rel * max(1.0, float(np.max(np.abs(vals))))
        Ls = []
        for sgn in (1.0, -1.0):
            q = copy.copy(prob)
            if dense:
                setattr(q, attr, base + sgn * h * d)
            else:
                M = base.copy()
                M.data = base.data + sgn * h * d
                setattr(q, attr, M)
            Ls.append(_loss(q, st, xref)[0])
        fd = (Ls[0] - Ls[1]) / (2.0 * h)
        an = float(g[key] @ d)
        assert abs(fd - an) <= rtol * abs(an), (key, fd, an)


GROUPS = [("dc", "c"), ("db", "b"), ("dh", "h"), ("dP", "P"), ("dA", "A"), ("dG", "G")]


def test_adjoint_matches_finite_differences_on_an_orthant_qp():
    _fd_check(dense_qp(seed=0), tol=1e-11, h_rel=1e-6, rtol=1e-5, groups=GROUPS)


def test_adjoint_matches_finite_differences_with_an_active_soc():
    # portfolio: long-only orthant + one active risk cone Q^6
    _fd_check(portfolio_socp(n=50, k=5, seed=0), tol=1e-9, h_rel=1e-5, rtol=1e-2, groups=GROUPS)


def test_adjoint_reduces_to_the_equality_qp_closed_form():
    prob = dense_qp(seed=1)
    prob = copy.copy(prob)
    prob.h = prob.h + 1e3  # every inequality row inactive
    r = ipm.solve(prob, ipm.Settings(abstol=1e-11, reltol=1e-11))
    assert r.status == "solved"
    xref = np.zeros(prob.n)
    gx = 2.0 * (r.x - xref)
    g = adjoint.backward(prob, r, gx)
    n, p = prob.n, prob.p
    Pf = kktmod.sym_from_upper(prob.P).toarray()
    A = prob.A.toarray()
    M = np.block([[Pf, A.T], [A, np.zeros((p, p))]])
    v0 = np.linalg.solve(M, np.concatenate([gx, np.zeros(p)]))
    scale = max(1.0, np.max(np.abs(v0)))
    assert np.max(np.abs(g["dc"] + v0[:n])) <= 1e-6 * scale
    assert np.max(np.abs(g["db"] - v0[n:])) <= 1e-6 * scale
    assert np.max(np.abs(g["dh"])) <= 1e-6 * scale
