"""Leaf groups: a large front whose many childless children share their update rows (the
arrowhead border of the portfolio SOCP: 20000 assets, each eliminated with its orthant
row, all updating the 201 rows of the risk cone and the budget).  Their pivots are
factored one warp per member and the parent receives −Σ L21·D·L21ᵀ as one split-K
product; the factor must still reconstruct the permuted KKT matrix, and the solve match
the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import cones as oc
from oracle import ipm
from oracle import kkt as ok
from workloads import portfolio_socp, random_cone_iterate
from _gpu_util import assert_certificate, rel_inf

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda()


def test_leaf_group_factor_reconstructs_the_matrix():
    import paper_2603_29197_gb300 as q
    # k = 170: the border (k + 1 cone rows + budget) makes the parent a large front (≥ 160)
    prob = portfolio_socp(n=600, k=170, seed=2)
    s, z, _, _ = random_cone_iterate(prob.l, prob.q, seed=5, scale_spread=1.0)
    S = q.Solver(prob)
    assert S.info()["large_fronts"] >= 1
    S.kkt_factor_at(T(s), T(z))
    perm, L, D = S.factor_dense()
    W = oc.NTScaling(s, z, prob.l, prob.q)
    Ke = (ok.assemble(prob, ok.z_block(W, prob.m)) + sp.diags(1e-8 * ok.reg_signs(prob))).toarray()
    Kp = Ke[np.ix_(perm, perm)]
    R = (L * D) @ L.T
    assert np.max(np.abs(R - Kp)) <= 1e-11 * np.abs(Kp).max() * max(1.0, np.abs(L).max()) ** 2
    S.close()


@pytest.mark.parametrize("mixed", [0, 1])
def test_leaf_group_solve_matches_oracle(mixed):
    import paper_2603_29197_gb300 as q
    prob = portfolio_socp(n=3000, k=170, seed=3)
    ref = ipm.solve(prob)
    assert ref.status == "solved"
    S = q.Solver(prob, mixed_precision=mixed)
    assert S.solve() == 0
    sol = S.solution()
    assert abs(sol["info"]["pobj"] - ref.pobj) <= 1e-6 * max(1.0, abs(ref.pobj))
    assert rel_inf(sol["x"], ref.x) <= 1e-5
    assert rel_inf(sol["z"], ref.z) <= 1e-5
    assert_certificate(prob, sol)
    S.close()
