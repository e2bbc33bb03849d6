"""Adjoint of the solution map (oracle; test infrastructure).

The paper has no adjoint; it is one of the forms grown beyond the plain solver, defined
here by implicit differentiation of the optimality conditions that the interior-point
method solves (eq. (1) with the KKT system of eq. (2)):

    F_x = Px + c + Aᵀy + Gᵀz = 0,   F_y = Ax − b = 0,   F_z = Gx + s − h = 0,

with the complementarity linearised exactly in the cone's Jordan algebra at the final
iterate (s, z):  z ∘ ds + s ∘ dz = 0,  i.e.  ds = B dz,  B = −Arw(z)⁻¹ Arw(s), where
Arw(u) is the arrow matrix of u (diag(u) on the orthant; [[u₀, u₁ᵀ], [u₁, u₀I]] on a
second-order cone).  With u = (x, y, z) this gives  K̂ du = −∂_θF dθ,

         [ P   Aᵀ   Gᵀ ]
    K̂ =  [ A   0    0  ]      (eq. (2)'s matrix with B in place of −WᵀW),
         [ G   0    B  ]

and for a loss L with g = ∂L/∂u:  v = K̂⁻ᵀ g,  dL = vᵀ K̂ du, so

    ∂L/∂c = −v_x,   ∂L/∂b = v_y,   ∂L/∂h = v_z,
    ∂L/∂A_rc = −(y_r v_x,c + v_y,r x_c),   ∂L/∂G_rc = −(z_r v_x,c + v_z,r x_c),
    ∂L/∂P_ij (stored upper entry i < j, both P_ij and P_ji move) = −(v_x,i x_j + v_x,j x_i),
    ∂L/∂P_ii = −v_x,i x_i.

On the central path B equals the NT block −W² in the limit; off it the two differ, and
only B matches finite differences of the solution map (an active second-order cone
showed a 1–2 % gap with −W²).  The linear solve is a library one: dense LU (numpy) up to
DENSE_MAX unknowns, sparse LU (SuperLU) beyond; Arw(z)⁻¹ is a library inverse per cone.

Pins (tests/test_oracle_adjoint.py): central finite differences of the oracle solve run
to tight tolerances, and the closed form of an equality-constrained QP whose inequality
rows are inactive, where the gradient follows from the reduced system [[P, Aᵀ], [A, 0]].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import kkt as kktmod

DENSE_MAX = 4000


def arrow(u):
    """Arw(u) for one second-order-cone block u = (u₀, u₁)."""
    d = len(u)
    M = np.zeros((d, d))
    M[0, :] = u
    M[:, 0] = u
    M[np.arange(1, d), np.arange(1, d)] = u[0]
    return M


def complementarity_block(s, z, l, q):
    """B = −Arw(z)⁻¹ Arw(s), block diagonal over the cones (sparse m×m)."""
    parts = []
    if l:
        parts.append(sp.diags(-s[:l] / z[:l]))
    o = l
    for d in q:
        parts.append(sp.csc_matrix(-np.linalg.inv(arrow(z[o:o + d])) @ arrow(s[o:o + d])))
        o += d
    if not parts:
        return sp.csc_matrix((0, 0))
    return sp.block_diag(parts, format="csc")


def kkt_hat(prob, s, z):
    """K̂: eq. (2)'s matrix with the exact complementarity block B in the z-z position."""
    n, p, m = prob.n, prob.p, prob.m
    Pf = kktmod.sym_from_upper(prob.P)
    A = prob.A if p else sp.csc_matrix((0, n))
    B = complementarity_block(s, z, prob.l, list(prob.q))
    return sp.bmat([[Pf, A.T, prob.G.T],
                    [A, sp.csc_matrix((p, p)) if p else None, None],
                    [prob.G, None, B if m else None]], format="csc")


def solve_transposed(K, g):
    """v = K⁻ᵀ g with a library LU (dense below DENSE_MAX unknowns)."""
    Kt = sp.csc_matrix(K.T)
    if Kt.shape[0] <= DENSE_MAX:
        return np.linalg.solve(Kt.toarray(), g)
    return spla.splu(Kt).solve(g)


def backward(prob, res, gx, gy=None, gz=None):
    """Gradients of L with respect to the problem data, given g = ∂L/∂(x, y, z) at the
    oracle's result `res` (ipm.Result: x, s, y, z).  Returns a dict with dP (values on
    P's stored upper pattern, CSC order), dc, dA (A's CSC order), db, dG (G's CSC
    order), dh, and v."""
    n, p, m = prob.n, prob.p, prob.m
    g = np.concatenate([np.asarray(gx, float),
                        np.zeros(p) if gy is None else np.asarray(gy, float),
                        np.zeros(m) if gz is None else np.asarray(gz, float)])
    v = solve_transposed(kkt_hat(prob, res.s, res.z), g)
    vx, vy, vz = v[:n], v[n:n + p], v[n + p:]
    x, y, z = res.x, res.y, res.z

    def per_entry(M, fn):
        M = sp.csc_matrix(M)
        out = np.zeros(M.nnz)
        for col in range(M.shape[1]):
            for k in range(M.indptr[col], M.indptr[col + 1]):
                out[k] = fn(M.indices[k], col)
        return out

    dP = per_entry(prob.P, lambda i, j: -vx[i] * x[i] if i == j else -(vx[i] * x[j] + vx[j] * x[i]))
    dA = per_entry(prob.A, lambda r, c: -(y[r] * vx[c] + vy[r] * x[c])) if p else np.zeros(0)
    dG = per_entry(prob.G, lambda r, c: -(z[r] * vx[c] + vz[r] * x[c]))
    return dict(dP=dP, dc=-vx, dA=dA, db=vy.copy(), dG=dG, dh=vz.copy(), v=v)
