"""Seeded synthetic instances of the problem class

    minimise ½xᵀPx + cᵀx   s.t.   Gx ⪯_K h,  Ax = b            (paper §1, eq. (1))

with K = (orthant of dimension l) × Q^{q_1} × … × Q^{q_nsoc}.  G's rows are ordered
orthant rows first, then the second-order-cone blocks in the order of ``q``; a vector
u is in Q^q when u_0 ≥ ‖u_{1:}‖.  P is stored as its upper triangle (paper §3 counts
"the upper half of P").

The instances stand in for the paper's benchmark families (§3.1: Huber, portfolio,
multi-period portfolio, group lasso, TV denoising), whose generators and images are
not available: each one reproduces the *shape* of a workload (sizes, sparsity
pattern, cone mix), never its data.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


@dataclass
class Problem:
    """Problem data in the layout the C-ABI takes (CSC, 0-based, sorted rows)."""

    n: int
    m: int
    p: int
    P: sp.csc_matrix  # n×n, upper triangle incl. diagonal
    c: np.ndarray
    A: sp.csc_matrix  # p×n
    b: np.ndarray
    G: sp.csc_matrix  # m×n
    h: np.ndarray
    l: int
    q: list = field(default_factory=list)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nsoc(self) -> int:
        return len(self.q)

    def size(self) -> int:
        """nnz(A) + nnz(G) + nnz(triu P): the size measure of the paper's Table 1 (§3)."""
        return int(self.A.nnz + self.G.nnz + self.P.nnz)

    def kkt_dim(self) -> int:
        return self.n + self.p + self.m


def _csc(M) -> sp.csc_matrix:
    M = sp.csc_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    M.eliminate_zeros()
    return M


def _finish(n, m, p, P, c, A, b, G, h, l, q, name, **meta) -> Problem:
    P = _csc(sp.triu(sp.csc_matrix(P)))
    A = _csc(A) if A is not None else sp.csc_matrix((0, n))
    G = _csc(G)
    assert P.shape == (n, n) and A.shape == (p, n) and G.shape == (m, n)
    assert l + int(sum(q)) == m
    return Problem(n=n, m=m, p=p, P=P, c=np.asarray(c, float), A=A,
                   b=np.asarray(b, float), G=G, h=np.asarray(h, float),
                   l=int(l), q=[int(v) for v in q], name=name, meta=meta)


# ---------------------------------------------------------------------------
# C1: plain sparse QP (n=200, p=50, m=l=400)
# ---------------------------------------------------------------------------
def dense_qp(n=200, p=50, m=400, rank=20, density=0.05, seed=0) -> Problem:
    """P = MMᵀ + 0.1 I (M n×rank N(0,1)); A, G iid Bernoulli(density) pattern with
    N(0,1) values, resampled until every row is nonzero and A has full row rank;
    x0 ~ N(0,1), s0 ~ U(0.5, 1.5), b = A x0, h = G x0 + s0, c ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, rank))
    P = M @ M.T + 0.1 * np.eye(n)

    def sparse_rows(rows):
        while True:
            mask = rng.random((rows, n)) < density
            vals = rng.standard_normal((rows, n))
            D = np.where(mask, vals, 0.0)
            if rows and np.all(mask.any(axis=1)):
                return D
            if rows == 0:
                return D

    while True:
        A = sparse_rows(p)
        if p == 0 or np.linalg.matrix_rank(A) == p:
            break
    G = sparse_rows(m)
    x0 = rng.standard_normal(n)
    s0 = rng.uniform(0.5, 1.5, m)
    b = A @ x0
    h = G @ x0 + s0
    c = rng.standard_normal(n)
    return _finish(n, m, p, P, c, A, b, G, h, m, [], f"dense_qp_n{n}", seed=seed)


# ---------------------------------------------------------------------------
# C2: minimum-fuel trajectory SOCP (double integrator, N steps)
# ---------------------------------------------------------------------------
def trajectory_socp(N=20000, horizon=200.0, state_cost=1e-3, pos_box=1e3, umax=1.0,
                    seed=0) -> Problem:
    """Minimum-fuel 3-D double-integrator trajectory over `horizon` seconds, dt = horizon/N
    (N = 20000 gives dt = 0.01).

    Variables, interleaved by stage: [x_0,u_0,σ_0, x_1,u_1,σ_1, …, x_{N-1},u_{N-1},σ_{N-1}, x_N]
    with x_k ∈ R⁶ (position, velocity), u_k ∈ R³, σ_k ∈ R.
    Objective Σ σ_k + state_cost·Σ‖x_k‖² (P diagonal).
    Equalities (stage order): x_0 = x_init; x_{k+1} = A_d x_k + B_d u_k; x_N = 0.
    Orthant rows (7 per stage): σ_k ≤ umax, ±position_k ≤ pos_box.
    SOCs (one Q⁴ per stage): (σ_k, u_k) ∈ Q⁴, i.e. ‖u_k‖ ≤ σ_k.
    x_init: position U(−100, 100) per axis, velocity 0.
    """
    rng = np.random.default_rng(seed)
    dt = horizon / N
    I3 = np.eye(3)
    Ad = np.block([[I3, dt * I3], [np.zeros((3, 3)), I3]])
    Bd = np.vstack([0.5 * dt * dt * I3, dt * I3])
    ns = 10
    n = ns * N + 6
    xoff = lambda k: ns * k  # noqa: E731
    uoff = lambda k: ns * k + 6  # noqa: E731
    soff = lambda k: ns * k + 9  # noqa: E731

    # P (diagonal): 2*state_cost on every state entry
    pd = np.zeros(n)
    for k in range(N + 1):
        pd[xoff(k):xoff(k) + 6] = 2.0 * state_cost
    P = sp.diags(pd).tocsc()
    c = np.zeros(n)
    c[[soff(k) for k in range(N)]] = 1.0

    x_init = np.concatenate([rng.uniform(-100.0, 100.0, 3), np.zeros(3)])

    # equality rows
    p = 6 * N + 12
    rows, cols, vals = [], [], []
    b = np.zeros(p)
    r = 0
    for i in range(6):  # x_0 = x_init
        rows.append(r + i); cols.append(xoff(0) + i); vals.append(1.0)
    b[0:6] = x_init
    r += 6
    Ad_nz = np.nonzero(Ad)
    Bd_nz = np.nonzero(Bd)
    for k in range(N):  # x_{k+1} - Ad x_k - Bd u_k = 0
        for i in range(6):
            rows.append(r + i); cols.append(xoff(k + 1) + i); vals.append(1.0)
        for i, j in zip(*Ad_nz):
            rows.append(r + i); cols.append(xoff(k) + j); vals.append(-Ad[i, j])
        for i, j in zip(*Bd_nz):
            rows.append(r + i); cols.append(uoff(k) + j); vals.append(-Bd[i, j])
        r += 6
    for i in range(6):  # x_N = 0
        rows.append(r + i); cols.append(xoff(N) + i); vals.append(1.0)
    r += 6
    A = sp.csc_matrix((vals, (rows, cols)), shape=(p, n))

    # cone rows: orthant (7 per stage) then SOCs (4 per stage)
    l = 7 * N
    m = l + 4 * N
    rows, cols, vals = [], [], []
    h = np.zeros(m)
    r = 0
    for k in range(N):
        rows.append(r); cols.append(soff(k)); vals.append(1.0); h[r] = umax; r += 1
        for i in range(3):
            rows.append(r); cols.append(xoff(k) + i); vals.append(1.0); h[r] = pos_box; r += 1
            rows.append(r); cols.append(xoff(k) + i); vals.append(-1.0); h[r] = pos_box; r += 1
    for k in range(N):
        rows.append(r); cols.append(soff(k)); vals.append(-1.0); r += 1
        for i in range(3):
            rows.append(r); cols.append(uoff(k) + i); vals.append(-1.0); r += 1
    G = sp.csc_matrix((vals, (rows, cols)), shape=(m, n))
    return _finish(n, m, p, P, c, A, b, G, h, l, [4] * N, f"trajectory_socp_N{N}",
                   seed=seed, N=N, dt=dt, x_init=x_init)


# ---------------------------------------------------------------------------
# C3: lasso as a QP with auxiliaries
# ---------------------------------------------------------------------------
def lasso_qp(rows=50000, cols=100000, density=1e-3, support=0.05, noise=0.01,
             lam_frac=0.1, seed=0) -> Problem:
    """min ½‖r‖² + λ·1ᵀt  s.t.  r − F x = −y,  x − t ≤ 0,  −x − t ≤ 0.

    Variables (x ∈ R^cols, t ∈ R^cols, r ∈ R^rows).  F has an iid pattern of the given
    density (sampled positions, duplicates merged) with N(0,1) values; x* has a
    `support` fraction of N(0,1) entries; y = F x* + noise·N(0,1); λ = lam_frac·‖Fᵀy‖∞.
    """
    rng = np.random.default_rng(seed)
    nnz = int(rng.binomial(rows * cols, density))
    lin = np.unique(rng.integers(0, rows * cols, size=nnz, dtype=np.int64))
    fr = (lin % rows).astype(np.int64)
    fc = (lin // rows).astype(np.int64)
    F = sp.csc_matrix((rng.standard_normal(lin.size), (fr, fc)), shape=(rows, cols))
    xs = np.zeros(cols)
    supp = rng.choice(cols, max(1, int(support * cols)), replace=False)
    xs[supp] = rng.standard_normal(supp.size)
    y = F @ xs + noise * rng.standard_normal(rows)
    lam = lam_frac * np.max(np.abs(F.T @ y))

    n = 2 * cols + rows
    Pd = np.concatenate([np.zeros(2 * cols), np.ones(rows)])
    P = sp.diags(Pd).tocsc()
    c = np.concatenate([np.zeros(cols), lam * np.ones(cols), np.zeros(rows)])
    I_c = sp.identity(cols, format="csc")
    A = sp.hstack([-F, sp.csc_matrix((rows, cols)), sp.identity(rows, format="csc")]).tocsc()
    b = -y
    G = sp.vstack([sp.hstack([I_c, -I_c, sp.csc_matrix((cols, rows))]),
                   sp.hstack([-I_c, -I_c, sp.csc_matrix((cols, rows))])]).tocsc()
    h = np.zeros(2 * cols)
    return _finish(n, 2 * cols, rows, P, c, A, b, G, h, 2 * cols, [],
                   f"lasso_qp_{rows}x{cols}", seed=seed, lam=lam, F=F, y=y,
                   rows=rows, cols=cols)


# ---------------------------------------------------------------------------
# C4: robust long-only portfolio with one factor-risk SOC
# ---------------------------------------------------------------------------
def _waterfill(d, mu, iters=200):
    """argmin Σ d_i x_i² − μᵀx  s.t. 1ᵀx = 1, x ≥ 0, by bisection on the multiplier
    (used only to place the risk cone so that it is active)."""
    lo, hi = mu.min() - 2.0 * d.max() * 2.0, mu.max()
    for _ in range(iters):
        nu = 0.5 * (lo + hi)
        s = np.maximum(0.0, (mu - nu) / (2.0 * d)).sum()
        if s > 1.0:
            lo = nu
        else:
            hi = nu
    nu = 0.5 * (lo + hi)
    return np.maximum(0.0, (mu - nu) / (2.0 * d))


def portfolio_socp(n=20000, k=200, gamma_frac=0.5, seed=0) -> Problem:
    """min xᵀDx − μᵀx  s.t.  1ᵀx = 1,  x ≥ 0,  ‖Fᵀx‖ ≤ γ.

    F n×k with N(0, 0.1²) entries, d_i ~ U(0.01, 0.1) (P = diag(2d)), μ_i ~ N(0.05, 0.02²).
    The SOC block is (γ, Fᵀx) ∈ Q^{k+1}: G rows [0; −Fᵀ], h = [γ; 0].  γ is
    gamma_frac·‖Fᵀx_u‖ where x_u solves the problem without the risk cone, so the cone
    is active at the solution.
    """
    rng = np.random.default_rng(seed)
    F = 0.1 * rng.standard_normal((n, k))
    d = rng.uniform(0.01, 0.1, n)
    mu = rng.normal(0.05, 0.02, n)
    xu = _waterfill(d, mu)
    gamma = gamma_frac * float(np.linalg.norm(F.T @ xu))
    P = sp.diags(2.0 * d).tocsc()
    c = -mu
    A = sp.csc_matrix(np.ones((1, n)))
    b = np.ones(1)
    G = sp.vstack([-sp.identity(n, format="csc"),
                   sp.csc_matrix((1, n)),
                   sp.csc_matrix(-F.T)]).tocsc()
    h = np.concatenate([np.zeros(n), [gamma], np.zeros(k)])
    return _finish(n, n + k + 1, 1, P, c, A, b, G, h, n, [k + 1],
                   f"portfolio_socp_n{n}", seed=seed, gamma=gamma, F=F, d=d, mu=mu)


# ---------------------------------------------------------------------------
# C5: batched small MPC SOCPs
# ---------------------------------------------------------------------------
def mpc_instance(T, A, B, x0, box=5.0, umax=1.0, ru=0.1) -> Problem:
    """One MPC instance: variables (x_1..x_T ∈ R^4, u_0..u_{T-1} ∈ R^2), interleaved
    per stage as [u_0, x_1, u_1, x_2, …, u_{T-1}, x_T];
    min Σ‖x_k‖² + ru·Σ‖u_k‖²  s.t.  x_{k+1} = A x_k + B u_k (x_0 given),
    |x_k| ≤ box (8 orthant rows per stage), (umax, u_k) ∈ Q³ per stage."""
    nx, nu = A.shape[0], B.shape[1]
    ns = nx + nu
    n = ns * T
    uoff = lambda k: ns * k  # noqa: E731
    xoff = lambda k: ns * k + nu  # noqa: E731  (x_{k+1})
    pd = np.zeros(n)
    for k in range(T):
        pd[uoff(k):uoff(k) + nu] = 2.0 * ru
        pd[xoff(k):xoff(k) + nx] = 2.0
    P = sp.diags(pd).tocsc()
    c = np.zeros(n)
    p = nx * T
    rows, cols, vals = [], [], []
    b = np.zeros(p)
    for k in range(T):  # x_{k+1} - A x_k - B u_k = 0
        r = nx * k
        for i in range(nx):
            rows.append(r + i); cols.append(xoff(k) + i); vals.append(1.0)
            for j in range(nu):
                rows.append(r + i); cols.append(uoff(k) + j); vals.append(-B[i, j])
            if k > 0:
                for j in range(nx):
                    rows.append(r + i); cols.append(xoff(k - 1) + j); vals.append(-A[i, j])
        if k == 0:
            b[0:nx] = A @ x0
    Aeq = sp.csc_matrix((vals, (rows, cols)), shape=(p, n))
    l = 2 * nx * T
    m = l + (nu + 1) * T
    rows, cols, vals = [], [], []
    h = np.zeros(m)
    r = 0
    for k in range(T):
        for i in range(nx):
            rows.append(r); cols.append(xoff(k) + i); vals.append(1.0); h[r] = box; r += 1
            rows.append(r); cols.append(xoff(k) + i); vals.append(-1.0); h[r] = box; r += 1
    for k in range(T):
        h[r] = umax; r += 1
        for j in range(nu):
            rows.append(r); cols.append(uoff(k) + j); vals.append(-1.0); r += 1
    G = sp.csc_matrix((vals, (rows, cols)), shape=(m, n))
    return _finish(n, m, p, P, c, Aeq, b, G, h, l, [nu + 1] * T, f"mpc_T{T}",
                   T=T, Adyn=A, Bdyn=B, x0=x0)


def mpc_batch(count=4096, tmin=10, tmax=60, nx=4, nu=2, seed=0):
    """`count` instances with horizons T ~ U{tmin..tmax}; A = Q diag(ρ) Qᵀ with Q Haar
    orthogonal and ρ ~ U(0.8, 0.99); B ~ N(0, 1/4); x0 ~ U(−1, 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        T = int(rng.integers(tmin, tmax + 1))
        Z = rng.standard_normal((nx, nx))
        Q, R = np.linalg.qr(Z)
        Q = Q * np.sign(np.diag(R))
        A = Q @ np.diag(rng.uniform(0.8, 0.99, nx)) @ Q.T
        B = 0.5 * rng.standard_normal((nx, nu))
        x0 = rng.uniform(-1.0, 1.0, nx)
        out.append(mpc_instance(T, A, B, x0))
    return out


# ---------------------------------------------------------------------------
# random interior iterates for cone-kernel parity
# ---------------------------------------------------------------------------
def random_cone_iterate(l, q, seed=0, margin=(0.05, 2.0), scale_spread=0.0):
    """Random strictly interior points s, z of K = R^l_+ × Q^{q_1} × …, and random
    directions ds, dz.  `scale_spread` > 0 draws per-cone magnitudes 10^U(−spread, spread)
    to imitate iterates near the end of an interior-point run."""
    rng = np.random.default_rng(seed)

    def point():
        parts = []
        if l:
            mag = 10.0 ** rng.uniform(-scale_spread, scale_spread, l)
            parts.append(mag * rng.uniform(*margin, l))
        for qk in q:
            mag = 10.0 ** rng.uniform(-scale_spread, scale_spread)
            u1 = rng.standard_normal(qk - 1)
            u0 = np.linalg.norm(u1) + rng.uniform(*margin)
            parts.append(mag * np.concatenate([[u0], u1]))
        return np.concatenate(parts) if parts else np.zeros(0)

    s = point()
    z = point()
    m = l + int(sum(q))
    ds = rng.standard_normal(m)
    dz = rng.standard_normal(m)
    return s, z, ds, dz
