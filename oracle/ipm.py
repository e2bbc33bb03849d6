"""Primal–dual interior-point method with NT scaling and Mehrotra predictor–corrector
(oracle; test infrastructure).

The paper (§2) states the structure of one iteration — two solves with one KKT
matrix (eq. (2)), factored once (§2.2), plus cone operations (§2.1) — and the
tolerances ε_abs = ε_rel = 1e-7 (§3).  It defers the method itself to QOCO and to
the CVXOPT notes (§1).  Every constant below that the paper does not print is a
reading of that method (an NT-scaled Mehrotra predictor–corrector):

  initial point   solve eq. (2) with W = I and rhs (−c, b, h); s = −z; shift s and z
                  into the cone (cones.shift_into_cone)
  residuals       r_x = Px + c + Aᵀy + Gᵀz,  r_y = Ax − b,  r_z = Gx + s − h
  stopping        ‖r_y‖∞ ≤ ε_abs + ε_rel·max(‖Ax‖∞, ‖b‖∞)
                  ‖r_z‖∞ ≤ ε_abs + ε_rel·max(‖Gx‖∞, ‖s‖∞, ‖h‖∞)
                  ‖r_x‖∞ ≤ ε_abs + ε_rel·max(‖Px‖∞, ‖Aᵀy‖∞, ‖Gᵀz‖∞, ‖c‖∞)
                  |sᵀz|  ≤ ε_abs + ε_rel·max(1, |pobj|, |dobj|)
  directions      K_ε[Δx; Δy; Δz] = [−r_x; −r_y; −r_z − W(λ\\d_s)],
                  Δs = W(λ\\d_s − WΔz)
                  affine     d_s = −λ∘λ
                  combined   d_s = −λ∘λ − (W⁻¹Δs_a)∘(WΔz_a) + σμe
  centring        μ = sᵀz/ν (ν = l + nsoc), σ = (1 − α_a)³
  steps           α_a = min(1, α_max(affine));  α = min(1, 0.99·α_max(combined))
  regularisation  ε = 1e-8 static; refinement to backward error 1e-10, ≤ 10 steps
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import cones
from . import kkt as kktmod


@dataclass
class Settings:
    abstol: float = 1e-7
    reltol: float = 1e-7
    abstol_inacc: float = 1e-5
    reltol_inacc: float = 1e-5
    max_iter: int = 200
    static_reg: float = 1e-8
    max_refine: int = 10
    refine_tol: float = 1e-10
    step_fraction: float = 0.99
    sigma_exponent: float = 3.0
    verbose: bool = False


@dataclass
class Result:
    status: str
    iters: int
    x: np.ndarray
    s: np.ndarray
    y: np.ndarray
    z: np.ndarray
    pobj: float
    dobj: float
    history: list = field(default_factory=list)


def _inf(v):
    return float(np.max(np.abs(v))) if v.size else 0.0


def residuals(prob, Pf, x, s, y, z):
    """r_x, r_y, r_z and the norms that scale the stopping tests."""
    Px = Pf @ x
    Aty = prob.A.T @ y if prob.p else np.zeros(prob.n)
    Gtz = prob.G.T @ z
    Ax = prob.A @ x if prob.p else np.zeros(0)
    Gx = prob.G @ x
    rx = Px + prob.c + Aty + Gtz
    ry = Ax - prob.b
    rz = Gx + s - prob.h
    xPx = float(x @ Px)
    pobj = 0.5 * xPx + float(prob.c @ x)
    dobj = -0.5 * xPx - float(prob.b @ y) - float(prob.h @ z)
    scale = dict(Px=_inf(Px), Aty=_inf(Aty), Gtz=_inf(Gtz), Ax=_inf(Ax), Gx=_inf(Gx))
    return rx, ry, rz, pobj, dobj, scale


def converged(prob, rx, ry, rz, gap, pobj, dobj, scale, s, abstol, reltol):
    ok_y = _inf(ry) <= abstol + reltol * max(scale["Ax"], _inf(prob.b))
    ok_z = _inf(rz) <= abstol + reltol * max(scale["Gx"], _inf(s), _inf(prob.h))
    ok_x = _inf(rx) <= abstol + reltol * max(scale["Px"], scale["Aty"], scale["Gtz"],
                                              _inf(prob.c))
    ok_g = abs(gap) <= abstol + reltol * max(1.0, abs(pobj), abs(dobj))
    return ok_x and ok_y and ok_z and ok_g


def newton_direction(prob, W, ks, rx, ry, rz, ds):
    """One search direction for the Jordan-algebra right-hand side d_s: the solve of
    K_ε[Δx; Δy; Δz] = [−r_x; −r_y; −r_z − W(λ\\d_s)] with refinement (ks), then
    Δs = W(λ\\d_s − WΔz).  It satisfies the linearised Newton system
        PΔx + AᵀΔy + GᵀΔz = −r_x,   AΔx = −r_y,   GΔx + Δs = −r_z,
        λ∘(WΔz + W⁻¹Δs) = d_s."""
    n, p, l, q = prob.n, prob.p, prob.l, prob.q
    t = cones.jordan_division(W.lam, ds, l, q)
    rhs = np.concatenate([-rx, -ry, -rz - W.apply_W(t)])
    d = ks.solve(rhs)
    dx, dy, dz = d[:n], d[n:n + p], d[n + p:]
    dsv = W.apply_W(t - W.apply_W(dz))
    return dx, dy, dz, dsv


def solve(prob, settings: Settings | None = None) -> Result:
    st = settings or Settings()
    n, p, m, l, q = prob.n, prob.p, prob.m, prob.l, prob.q
    nu = cones.degree(l, q)
    e = cones.identity(l, q)
    Pf = kktmod.sym_from_upper(prob.P)
    signs = kktmod.reg_signs(prob)

    # --- initial point: eq. (2) with W = I, rhs (−c, b, h) ---
    K0 = kktmod.assemble(prob, kktmod.initial_W2(prob))
    ks = kktmod.KKTSolver(K0, signs, st.static_reg, st.max_refine, st.refine_tol)
    sol = ks.solve(np.concatenate([-prob.c, prob.b, prob.h]))
    x, y, z = sol[:n], sol[n:n + p], sol[n + p:]
    s = cones.shift_into_cone(-z, l, q)
    z = cones.shift_into_cone(z, l, q)

    history = []
    status = "max_iter"
    it = 0
    for it in range(st.max_iter + 1):
        rx, ry, rz, pobj, dobj, scale = residuals(prob, Pf, x, s, y, z)
        gap = float(s @ z)
        mu = gap / nu if nu else 0.0
        rec = dict(iter=it, pobj=pobj, dobj=dobj, gap=gap, pres=max(_inf(ry), _inf(rz)),
                   dres=_inf(rx))
        if converged(prob, rx, ry, rz, gap, pobj, dobj, scale, s, st.abstol, st.reltol):
            history.append(rec)
            status = "solved"
            break
        if it == st.max_iter:
            history.append(rec)
            if converged(prob, rx, ry, rz, gap, pobj, dobj, scale, s,
                         st.abstol_inacc, st.reltol_inacc):
                status = "solved_inaccurate"
            break

        # --- NT scaling and the KKT matrix of this iteration ---
        W = cones.NTScaling(s, z, l, q)
        lam = W.lam
        K = kktmod.assemble(prob, kktmod.z_block(W, m))
        ks = kktmod.KKTSolver(K, signs, st.static_reg, st.max_refine, st.refine_tol)

        def direction(ds):
            return newton_direction(prob, W, ks, rx, ry, rz, ds)

        # --- predictor (affine) ---
        lamlam = cones.jordan_product(lam, lam, l, q)
        dx_a, dy_a, dz_a, ds_a = direction(-lamlam)
        refine_a = ks.last_refine_steps
        alpha_a = min(1.0, cones.max_step(s, ds_a, l, q), cones.max_step(z, dz_a, l, q))
        sigma = (1.0 - alpha_a) ** st.sigma_exponent

        # --- corrector (combined) ---
        corr = cones.jordan_product(W.apply_Winv(ds_a), W.apply_W(dz_a), l, q)
        dx, dy, dz, dsv = direction(-lamlam - corr + sigma * mu * e)
        amax = min(cones.max_step(s, dsv, l, q), cones.max_step(z, dz, l, q))
        alpha = min(1.0, st.step_fraction * amax)

        x = x + alpha * dx
        y = y + alpha * dy
        z = z + alpha * dz
        s = s + alpha * dsv
        rec.update(alpha_a=alpha_a, sigma=sigma, alpha=alpha, refine_a=refine_a,
                   refine_c=ks.last_refine_steps, berr=ks.last_backward_error)
        history.append(rec)
        if st.verbose:
            print(f"{it:3d} pobj {pobj:+.6e} dobj {dobj:+.6e} gap {gap:.2e} "
                  f"pres {rec['pres']:.2e} dres {rec['dres']:.2e} a {alpha:.3f} s {sigma:.2e}")
        if not (np.all(np.isfinite(x)) and np.all(np.isfinite(s)) and math.isfinite(alpha)):
            status = "numerical_error"
            break

    rx, ry, rz, pobj, dobj, _ = residuals(prob, Pf, x, s, y, z)
    return Result(status=status, iters=it, x=x, s=s, y=y, z=z, pobj=pobj, dobj=dobj,
                  history=history)
