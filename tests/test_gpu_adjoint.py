"""Adjoint (qoco_gpu_backward) and parametric re-solve (qoco_gpu_update_data) through
the C ABI, against the oracle's adjoint (oracle/adjoint.py, pinned by finite
differences and closed forms in test_oracle_adjoint.py) and against properties that
hold at any size: the returned v = (−dc, db, dh) must satisfy K̂ᵀv = g for the
final iterate's exact complementarity block, and the data gradients must follow
from v and the solution entry by entry."""
import copy

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import adjoint, ipm
from workloads import dense_qp, mpc_instance, portfolio_socp, trajectory_socp
from _gpu_util import assert_certificate, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_2603_29197_gb300 as qq
    return qq


def _t(a):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda()


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def _mpc_small():
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    A = Q @ np.diag(rng.uniform(0.8, 0.99, 4)) @ Q.T
    B = rng.standard_normal((4, 2)) / 2.0
    return mpc_instance(T=25, A=A, B=B, x0=rng.uniform(-1, 1, 4) * 4.0)


CASES = {
    "dense_qp": lambda: dense_qp(seed=0),
    "portfolio_n200": lambda: portfolio_socp(n=200, k=20, seed=0),
    "mpc_T25": _mpc_small,
}
# The adjoint at an active second-order cone depends on how close the final iterate
# sits to the cone's boundary (Arw(z)⁻¹ is ill-conditioned there); the two solvers stop
# at slightly different iterates, so that case gets a looser bound.
TOL = {"dense_qp": 1e-6, "portfolio_n200": 2e-3, "mpc_T25": 2e-3}


def _gpu_grads(q, prob, xref):
    S = q.Solver(prob)
    assert S.solve() == 0
    sol = S.solution()
    g = S.backward(dx=_t(2.0 * (sol["x"] - xref)))
    return S, sol, _np(g)


@pytest.mark.parametrize("name", list(CASES))
def test_backward_matches_oracle_adjoint(q, name):
    prob = CASES[name]()
    xref = np.full(prob.n, 1.0 / prob.n)
    ref = ipm.solve(prob)
    assert ref.status == "solved"
    go = adjoint.backward(prob, ref, 2.0 * (ref.x - xref))
    S, sol, gg = _gpu_grads(q, prob, xref)
    bi = S.backward_info()
    assert bi["backward_error"] <= 1e-10, bi
    for k in ("dP", "dc", "dA", "db", "dG", "dh"):
        if go[k].size == 0:
            continue
        assert rel_inf(gg[k], go[k]) <= TOL[name], (k, rel_inf(gg[k], go[k]), bi)
    S.close()


def _khat_T_residual(prob, sol, v, g):
    """‖K̂ᵀv − g‖∞ / (‖K̂‖∞‖v‖∞ + ‖g‖∞), K̂ built with scipy from the data and the
    returned final iterate (independent of the GPU path)."""
    K = adjoint.kkt_hat(prob, sol["s"], sol["z"])
    r = K.T @ v - g
    nK = float(np.max(np.abs(K).sum(axis=1)))
    return float(np.max(np.abs(r)) / (nK * np.max(np.abs(v)) + np.max(np.abs(g))))


@pytest.mark.parametrize("name", list(CASES))
def test_backward_solves_the_exact_adjoint_system(q, name):
    prob = CASES[name]()
    xref = np.full(prob.n, 1.0 / prob.n)
    S, sol, gg = _gpu_grads(q, prob, xref)
    v = np.concatenate([-gg["dc"], gg["db"], gg["dh"]])
    g = np.concatenate([2.0 * (sol["x"] - xref), np.zeros(prob.p + prob.m)])
    assert _khat_T_residual(prob, sol, v, g) <= 1e-9
    S.close()


def _data_grads_from_v(prob, sol, v, sample, rng):
    """Entrywise data gradients from v and the solution (host formula), on a sample."""
    n, p = prob.n, prob.p
    x, y, z = sol["x"], sol["y"], sol["z"]
    vx, vy, vz = v[:n], v[n:n + p], v[n + p:]
    out = {}
    for key, M, fn in (("dP", prob.P, lambda i, j: -vx[i] * x[i] if i == j else -(vx[i] * x[j] + vx[j] * x[i])),
                       ("dA", prob.A, lambda r, c: -(y[r] * vx[c] + vy[r] * x[c])),
                       ("dG", prob.G, lambda r, c: -(z[r] * vx[c] + vz[r] * x[c]))):
        M = sp.csc_matrix(M)
        if M.nnz == 0:
            continue
        ks = rng.choice(M.nnz, size=min(sample, M.nnz), replace=False)
        cols = np.searchsorted(M.indptr, ks, side="right") - 1
        out[key] = (ks, np.array([fn(M.indices[k], c) for k, c in zip(ks, cols)]))
    return out


def test_backward_full_size_portfolio(q):
    """C4 at full size: n = 20000 assets, Q^201 risk cone, N_K = 40202."""
    prob = portfolio_socp(n=20000, k=200, seed=0)
    xref = np.full(prob.n, 1.0 / prob.n)
    S, sol, gg = _gpu_grads(q, prob, xref)
    v = np.concatenate([-gg["dc"], gg["db"], gg["dh"]])
    g = np.concatenate([2.0 * (sol["x"] - xref), np.zeros(prob.p + prob.m)])
    assert _khat_T_residual(prob, sol, v, g) <= 1e-9
    rng = np.random.default_rng(0)
    for key, (ks, want) in _data_grads_from_v(prob, sol, v, 2000, rng).items():
        got = gg[key][ks]
        assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want))), key
    S.close()


def test_backward_needs_a_completed_solve(q):
    from paper_2603_29197_gb300 import _lib
    prob = dense_qp(n=40, p=5, m=60, rank=5, density=0.2, seed=2)
    S = q.Solver(prob)
    with pytest.raises(q.SolverError) as e:
        S.backward(dx=_t(np.ones(prob.n)))
    assert e.value.code == _lib.ERR_NO_FACTOR
    assert S.solve() == 0
    S.backward(dx=_t(np.ones(prob.n)))
    S.update_data(c=prob.c)
    with pytest.raises(q.SolverError) as e:
        S.backward(dx=_t(np.ones(prob.n)))
    assert e.value.code == _lib.ERR_NO_FACTOR
    S.close()


# ---- parametric re-solve ---------------------------------------------------------

def _perturbed(prob, seed):
    rng = np.random.default_rng(seed)
    new = copy.copy(prob)
    new.c = prob.c + 0.1 * rng.standard_normal(prob.n)
    new.h = prob.h + 0.05 * np.abs(rng.standard_normal(prob.m))
    G = prob.G.copy()
    G.data = G.data * (1.0 + 0.05 * rng.standard_normal(G.nnz))
    new.G = G
    P = sp.csc_matrix(prob.P).copy()  # 1.1·P + 0.05·I stays positive semidefinite
    rows = P.indices
    cols = np.repeat(np.arange(P.shape[1]), np.diff(P.indptr))
    P.data = 1.1 * P.data + 0.05 * (rows == cols)
    new.P = P
    return new


@pytest.mark.parametrize("on_device", [False, True])
def test_update_data_matches_a_fresh_setup(q, on_device):
    prob = dense_qp(seed=3)
    new = _perturbed(prob, 1)
    S = q.Solver(prob)
    assert S.solve() == 0
    conv = _t if on_device else (lambda a: np.asarray(a, dtype=np.float64))
    S.update_data(P=conv(new.P.tocsc().data), c=conv(new.c), A=conv(new.A.tocsc().data), b=conv(new.b),
                  G=conv(new.G.tocsc().data), h=conv(new.h))
    assert S.solve() == 0
    a = S.solution()
    F = q.Solver(new)
    assert F.solve() == 0
    b = F.solution()
    assert a["info"]["iters"] == b["info"]["iters"]
    for k in ("x", "y", "z", "s"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-12)
    S.close()
    F.close()


@pytest.mark.parametrize("make", [lambda: dense_qp(seed=3), lambda: portfolio_socp(n=300, k=20, seed=2),
                                  lambda: trajectory_socp(N=150, seed=5)])
def test_update_data_resolve_matches_the_oracle_on_the_new_data(q, make):
    """A parametric re-solve (new values, same patterns; the symbolic analysis and every
    device buffer kept) reaches the oracle's solution of the perturbed problem: objective
    within 1e-6, x, y, z within 1e-5 (relative to max(1, ‖·‖∞)), and an independent KKT
    certificate of the new data."""
    prob = make()
    new = _perturbed(prob, 7)
    S = q.Solver(prob)
    assert S.solve() == 0
    S.update_data(P=new.P.tocsc().data, c=new.c, A=new.A.tocsc().data if prob.p else None,
                  b=new.b if prob.p else None, G=new.G.tocsc().data, h=new.h)
    assert S.solve() == 0
    a = S.solution()
    ref = ipm.solve(new)
    assert ref.status == "solved"
    assert abs(a["info"]["pobj"] - ref.pobj) <= 1e-6 * max(1.0, abs(ref.pobj))
    for k in ("x", "y", "z"):
        assert rel_inf(a[k], getattr(ref, k)) <= 1e-5, k
    assert_certificate(new, a)
    S.close()


def test_update_data_with_unchanged_values_is_bitwise_stable(q):
    prob = portfolio_socp(n=200, k=20, seed=1)
    S = q.Solver(prob)
    assert S.solve() == 0
    a = S.solution()
    S.update_data(P=prob.P.tocsc().data, c=prob.c, A=prob.A.tocsc().data, b=prob.b, G=prob.G.tocsc().data,
                  h=prob.h)
    assert S.solve() == 0
    b = S.solution()
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["z"], b["z"])
    S.close()


def test_update_data_rejects_non_finite_host_values(q):
    from paper_2603_29197_gb300 import _lib
    prob = dense_qp(n=40, p=5, m=60, rank=5, density=0.2, seed=2)
    S = q.Solver(prob)
    bad = prob.c.copy()
    bad[3] = np.nan
    with pytest.raises(q.SolverError) as e:
        S.update_data(c=bad)
    assert e.value.code == _lib.ERR_NONFINITE_DATA
    S.close()


def test_autograd_function_matches_backward_and_oracle(q):
    import torch
    prob = portfolio_socp(n=200, k=20, seed=0)
    S = q.Solver(prob)
    Fn = q.solve_function()
    leaves = [_t(a).requires_grad_(True) for a in (prob.P.tocsc().data, prob.c, prob.A.tocsc().data, prob.b,
                                                    prob.G.tocsc().data, prob.h)]
    x, y, z = Fn.apply(S, *leaves)
    xref = torch.full_like(x, 1.0 / prob.n)
    loss = ((x - xref) ** 2).sum()
    loss.backward()
    ref = ipm.solve(prob)
    go = adjoint.backward(prob, ref, 2.0 * (ref.x - 1.0 / prob.n))
    for leaf, key in zip(leaves, ("dP", "dc", "dA", "db", "dG", "dh")):
        assert rel_inf(leaf.grad.cpu().numpy(), go[key]) <= 2e-3, key
    S.close()
