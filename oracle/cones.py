"""Cone algebra on K = R^l_+ × Q^{q_1} × … × Q^{q_nsoc} (oracle; test infrastructure).

The paper names the cone operations its GPU backend parallelises — Jordan products,
projection onto K and the Nesterov–Todd scalings (§2.1, "Cone operations ...") — and
maps one thread to each cone (§2.3).  It does not print their formulas; it defers to
the QOCO and CVXOPT references (§1).  The formulas below are the standard Euclidean
Jordan algebra of the second-order cone and the NT construction of those notes,
written out per cone with plain loops.

Layout: a vector u ∈ R^m, m = l + Σq_k, holds the orthant part u[0:l] first, then
each SOC block in order; an SOC block is (u_0, u_1) with u_0 the scalar part, and
u ∈ Q^q  ⇔  u_0 ≥ ‖u_1‖.

Pins (tests/test_oracle_cones.py): Wz = W⁻¹s = λ, W² = η²(2w̄w̄ᵀ − J), w̄ᵀJw̄ = 1,
sᵀz = λᵀλ, λ∘(λ\\v) = v, e∘u = u, u∘v = v∘u; max step against bisection on cone
membership; projection against a brute-force minimiser and the Moreau decomposition.
"""
from __future__ import annotations

import math

import numpy as np


def blocks(l, q):
    """(start, dim) of each SOC block."""
    out, o = [], l
    for qk in q:
        out.append((o, int(qk)))
        o += int(qk)
    return out


def identity(l, q):
    """Jordan identity e: 1 on the orthant, (1, 0, …, 0) on each SOC."""
    e = np.zeros(l + int(sum(q)))
    e[:l] = 1.0
    for o, _ in blocks(l, q):
        e[o] = 1.0
    return e


def jordan_product(u, v, l, q):
    """u∘v: orthant elementwise; SOC (uᵀv, u_0 v_1 + v_0 u_1)."""
    w = np.empty_like(u)
    w[:l] = u[:l] * v[:l]
    for o, d in blocks(l, q):
        a, b = u[o:o + d], v[o:o + d]
        w[o] = float(np.dot(a, b))
        w[o + 1:o + d] = a[0] * b[1:] + b[0] * a[1:]
    return w


def jordan_division(lam, v, l, q):
    """w = λ\\v, the solution of λ∘w = v.

    SOC: w_0 = (λ_0 v_0 − λ_1ᵀv_1) / (λ_0² − ‖λ_1‖²),  w_1 = (v_1 − w_0 λ_1) / λ_0."""
    w = np.empty_like(v)
    w[:l] = v[:l] / lam[:l]
    for o, d in blocks(l, q):
        L, V = lam[o:o + d], v[o:o + d]
        det = L[0] * L[0] - float(np.dot(L[1:], L[1:]))
        w0 = (L[0] * V[0] - float(np.dot(L[1:], V[1:]))) / det
        w[o] = w0
        w[o + 1:o + d] = (V[1:] - w0 * L[1:]) / L[0]
    return w


def jnorm2(u):
    """uᵀJu = u_0² − ‖u_1‖² for one SOC block."""
    return u[0] * u[0] - float(np.dot(u[1:], u[1:]))


class NTScaling:
    """Nesterov–Todd scaling of (s, z) ∈ int K × int K.

    Orthant: W = diag(w), w_i = √(s_i/z_i), λ_i = √(s_i z_i).
    SOC block: s̄ = s/√(sᵀJs), z̄ = z/√(zᵀJz), γ = √((1 + s̄ᵀz̄)/2),
               w̄ = (s̄ + J z̄)/(2γ), η = (sᵀJs / zᵀJz)^{1/4},
               W = η [[w̄_0, w̄_1ᵀ], [w̄_1, I + w̄_1 w̄_1ᵀ/(1 + w̄_0)]],
               λ = W z,  W² = η² (2 w̄ w̄ᵀ − J).
    W is symmetric, so Wᵀ = W throughout.
    """

    def __init__(self, s, z, l, q):
        self.l, self.q = l, list(q)
        self.w = np.sqrt(s[:l] / z[:l])
        self.eta = []
        self.wbar = []
        for o, d in blocks(l, q):
            sb, zb = s[o:o + d], z[o:o + d]
            sj, zj = jnorm2(sb), jnorm2(zb)
            sbar = sb / math.sqrt(sj)
            zbar = zb / math.sqrt(zj)
            gamma = math.sqrt(0.5 * (1.0 + float(np.dot(sbar, zbar))))
            Jz = zbar.copy()
            Jz[1:] = -Jz[1:]
            self.wbar.append((sbar + Jz) / (2.0 * gamma))
            self.eta.append((sj / zj) ** 0.25)
        self.lam = self.apply_W(z)

    # dense blocks, for assembly and for the identity tests
    def W_block(self, k):
        wb, eta = self.wbar[k], self.eta[k]
        d = wb.size
        W = np.empty((d, d))
        W[0, 0] = wb[0]
        W[0, 1:] = wb[1:]
        W[1:, 0] = wb[1:]
        W[1:, 1:] = np.eye(d - 1) + np.outer(wb[1:], wb[1:]) / (1.0 + wb[0])
        return eta * W

    def Winv_block(self, k):
        wb, eta = self.wbar[k], self.eta[k]
        d = wb.size
        W = np.empty((d, d))
        W[0, 0] = wb[0]
        W[0, 1:] = -wb[1:]
        W[1:, 0] = -wb[1:]
        W[1:, 1:] = np.eye(d - 1) + np.outer(wb[1:], wb[1:]) / (1.0 + wb[0])
        return W / eta

    def W2_block(self, k):
        """W² = η²(2w̄w̄ᵀ − J) for SOC block k."""
        wb, eta = self.wbar[k], self.eta[k]
        J = -np.eye(wb.size)
        J[0, 0] = 1.0
        return eta * eta * (2.0 * np.outer(wb, wb) - J)

    def W2_orthant(self):
        return self.w * self.w

    def apply_W(self, v):
        out = np.empty_like(v)
        out[:self.l] = self.w * v[:self.l]
        for k, (o, d) in enumerate(blocks(self.l, self.q)):
            out[o:o + d] = self.W_block(k) @ v[o:o + d]
        return out

    def apply_Winv(self, v):
        out = np.empty_like(v)
        out[:self.l] = v[:self.l] / self.w
        for k, (o, d) in enumerate(blocks(self.l, self.q)):
            out[o:o + d] = self.Winv_block(k) @ v[o:o + d]
        return out


def max_step(u, du, l, q):
    """sup{α ≥ 0 : u + α du ∈ K} for u ∈ int K (may be +inf).

    Orthant: min over du_i < 0 of −u_i/du_i.
    SOC: with a = du_0² − ‖du_1‖², b = u_0 du_0 − u_1ᵀdu_1, c = u_0² − ‖u_1‖² > 0, the
    block leaves the cone at the smallest positive root of aα² + 2bα + c (none: +inf).
    """
    alpha = math.inf
    for i in range(l):
        if du[i] < 0.0:
            alpha = min(alpha, -u[i] / du[i])
    for o, d in blocks(l, q):
        U, D = u[o:o + d], du[o:o + d]
        a = D[0] * D[0] - float(np.dot(D[1:], D[1:]))
        b = U[0] * D[0] - float(np.dot(U[1:], D[1:]))
        c = U[0] * U[0] - float(np.dot(U[1:], U[1:]))
        alpha = min(alpha, _smallest_positive_root(a, b, c))
    return alpha


def _smallest_positive_root(a, b, c):
    """Smallest α > 0 with aα² + 2bα + c = 0, given c > 0; +inf if none."""
    if a == 0.0:
        return -c / (2.0 * b) if b < 0.0 else math.inf
    disc = b * b - a * c
    if disc < 0.0:
        return math.inf
    r = math.sqrt(disc)
    roots = [(-b - r) / a, (-b + r) / a]
    pos = [t for t in roots if t > 0.0]
    return min(pos) if pos else math.inf


def shift_into_cone(u, l, q):
    """Initial-point shift: α = max over cones of (−u_i) (orthant) or ‖u_1‖ − u_0 (SOC);
    if α < 0 return u, else u + (1 + α)e."""
    cand = [-u[i] for i in range(l)]
    for o, d in blocks(l, q):
        cand.append(float(np.linalg.norm(u[o + 1:o + d])) - u[o])
    alpha = max(cand) if cand else -1.0
    if alpha < 0.0:
        return u.copy()
    return u + (1.0 + alpha) * identity(l, q)


def project(u, l, q):
    """Euclidean projection onto K: orthant max(·,0); SOC
    u if ‖u_1‖ ≤ u_0, 0 if ‖u_1‖ ≤ −u_0, else ((u_0 + ‖u_1‖)/2)(1, u_1/‖u_1‖)."""
    out = u.copy()
    out[:l] = np.maximum(u[:l], 0.0)
    for o, d in blocks(l, q):
        u0, u1 = u[o], u[o + 1:o + d]
        t = float(np.linalg.norm(u1))
        if t <= u0:
            continue
        if t <= -u0:
            out[o:o + d] = 0.0
            continue
        f = 0.5 * (u0 + t)
        out[o] = f
        out[o + 1:o + d] = f * u1 / t
    return out


def in_cone(u, l, q, tol=0.0):
    """Membership test with slack tol (used by the bisection pin)."""
    if l and np.min(u[:l]) < -tol:
        return False
    for o, d in blocks(l, q):
        if u[o] - np.linalg.norm(u[o + 1:o + d]) < -tol:
            return False
    return True


def degree(l, q):
    """ν = l + nsoc, the degree of K (μ = sᵀz/ν)."""
    return l + len(q)
