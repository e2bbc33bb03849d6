"""The KKT system of each interior-point iteration (oracle; test infrastructure).

Paper §2.2, eq. (2): the coefficient matrix

        [ P   Aᵀ   Gᵀ     ]
    K = [ A   0    0      ]      (N_K = n + p + m)
        [ G   0   −WᵀW    ]

is factored once per iteration and solved twice.  Static regularisation is not in
the paper (it only says the matrix is factored by an LDLᵀ); we read it as the usual
quasidefinite form K_ε = K + ε·diag(+1 on x, −1 on y, −1 on z), which every
symmetric ordering factors without pivoting, and we refine each solve against the
unregularised K:  x ← x + K_ε⁻¹(r − Kx)  until the normwise backward error
‖Kx − r‖∞ / (‖K‖∞‖x‖∞ + ‖r‖∞) is below the target.

The solve uses a library sparse LU (SuperLU via scipy) of K_ε as the "K_ε⁻¹" step;
`dense_ldlt` is a plain textbook LDLᵀ used to pin the GPU factor on tiny cases.

Pins (tests/test_oracle_kkt.py): the solve against a dense numpy solve; the refined
backward error; dense_ldlt's reconstruction L D Lᵀ = K_ε and its agreement with a
Cholesky factor on positive-definite inputs.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cones


def sym_from_upper(U):
    """Full symmetric matrix from an upper triangle (incl. diagonal)."""
    U = sp.csc_matrix(U)
    return (U + sp.triu(U, 1).T).tocsc()


def z_block(scaling, m):
    """W² over the whole cone (block diagonal, m×m)."""
    l, q = scaling.l, scaling.q
    parts = []
    if l:
        parts.append(sp.diags(scaling.W2_orthant()))
    for k in range(len(q)):
        parts.append(sp.csc_matrix(scaling.W2_block(k)))
    if not parts:
        return sp.csc_matrix((m, m))
    return sp.block_diag(parts).tocsc()


def assemble(prob, W2):
    """K of eq. (2) with the given m×m W² block (W2 = identity for the initial point)."""
    n, p, m = prob.n, prob.p, prob.m
    Pf = sym_from_upper(prob.P)
    A = prob.A if p else sp.csc_matrix((0, n))
    K = sp.bmat([[Pf, A.T, prob.G.T],
                 [A, sp.csc_matrix((p, p)) if p else None, None],
                 [prob.G, None, -W2]], format="csc")
    return K


def reg_signs(prob):
    return np.concatenate([np.ones(prob.n), -np.ones(prob.p), -np.ones(prob.m)])


def regularise(K, signs, eps):
    return (K + sp.diags(eps * signs)).tocsc()


class KKTSolver:
    """Factor K_ε once; solve with refinement against K."""

    def __init__(self, K, signs, eps, max_refine=10, tol=1e-10):
        self.K = sp.csc_matrix(K)
        self.Keps = regularise(self.K, signs, eps)
        self.lu = spla.splu(self.Keps, permc_spec="MMD_AT_PLUS_A",
                            diag_pivot_thresh=0.0, options={"SymmetricMode": True})
        self.normK = float(abs(self.K).sum(axis=1).max()) if self.K.nnz else 0.0
        self.max_refine = max_refine
        self.tol = tol
        self.last_refine_steps = 0
        self.last_backward_error = 0.0

    def backward_error(self, x, r):
        res = r - self.K @ x
        den = self.normK * np.max(np.abs(x), initial=0.0) + np.max(np.abs(r), initial=0.0)
        return (np.max(np.abs(res), initial=0.0) / den) if den > 0 else 0.0

    def solve(self, r):
        x = self.lu.solve(r)
        steps = 0
        be = self.backward_error(x, r)
        while be > self.tol and steps < self.max_refine:
            x = x + self.lu.solve(r - self.K @ x)
            steps += 1
            be = self.backward_error(x, r)
        self.last_refine_steps = steps
        self.last_backward_error = be
        return x


def dense_ldlt(M, signs=None, dyn_thresh=1e-13, dyn_value=1e-7):
    """Textbook LDLᵀ without pivoting of a dense symmetric M (natural order):
    d_j = M_jj − Σ_{k<j} L_jk² d_k;  L_ij = (M_ij − Σ_{k<j} L_ik L_jk d_k)/d_j.
    With `signs`, a pivot whose signed value sign_j·d_j is below dyn_thresh is
    replaced by sign_j·dyn_value (dynamic regularisation)."""
    M = np.array(M, dtype=float)
    N = M.shape[0]
    L = np.eye(N)
    d = np.zeros(N)
    for j in range(N):
        d[j] = M[j, j] - np.sum(L[j, :j] ** 2 * d[:j])
        if signs is not None and signs[j] * d[j] < dyn_thresh:
            d[j] = signs[j] * dyn_value
        for i in range(j + 1, N):
            L[i, j] = (M[i, j] - np.sum(L[i, :j] * L[j, :j] * d[:j])) / d[j]
    return L, d


def initial_W2(prob):
    """W = I for the initial point."""
    return sp.identity(prob.m, format="csc")


def scaling_W2(scaling, m):
    return z_block(scaling, m)


__all__ = ["assemble", "reg_signs", "regularise", "KKTSolver", "dense_ldlt",
           "z_block", "sym_from_upper", "cones"]
