"""Helpers shared by the GPU parity tests (comparison metrics and a CPU KKT
certificate computed from the problem data and a returned solution)."""
import numpy as np


def rel_inf(a, b, floor=1.0):
    """‖a − b‖∞ / max(floor, ‖b‖∞)."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(floor, float(np.max(np.abs(b)))))


def blockwise_rel(a, b, l, q):
    """Largest per-cone relative difference (orthant entrywise, SOC blockwise)."""
    worst = 0.0
    if l:
        worst = max(worst, float(np.max(np.abs(a[:l] - b[:l]) / np.maximum(np.abs(b[:l]), 1e-300))))
    o = l
    for qk in q:
        nb = max(float(np.max(np.abs(b[o:o + qk]))), 1e-300)
        worst = max(worst, float(np.max(np.abs(a[o:o + qk] - b[o:o + qk]))) / nb)
        o += qk
    return worst


def kkt_certificate(prob, x, s, y, z):
    """Residual norms, cone membership margins and gap of (x, s, y, z) for the problem,
    computed with scipy from the data (independent of both solvers)."""
    Pu = prob.P
    Px = Pu @ x + Pu.T @ x - Pu.diagonal() * x
    rx = Px + prob.c + (prob.A.T @ y if prob.p else 0.0) + prob.G.T @ z
    ry = (prob.A @ x - prob.b) if prob.p else np.zeros(0)
    rz = prob.G @ x + s - prob.h
    def cone_margin(u):
        mins = [np.min(u[:prob.l])] if prob.l else []
        o = prob.l
        for qk in prob.q:
            mins.append(u[o] - np.linalg.norm(u[o + 1:o + qk]))
            o += qk
        return min(mins) if mins else 0.0
    pobj = 0.5 * x @ Px + prob.c @ x
    return dict(rx=float(np.max(np.abs(rx), initial=0)), ry=float(np.max(np.abs(ry), initial=0)),
                rz=float(np.max(np.abs(rz), initial=0)), s_margin=float(cone_margin(s)),
                z_margin=float(cone_margin(z)), gap=float(s @ z), pobj=float(pobj),
                scale=1.0 + max(float(np.max(np.abs(prob.c), initial=0)),
                                float(np.max(np.abs(prob.b), initial=0)),
                                float(np.max(np.abs(prob.h), initial=0))))


def assert_certificate(prob, sol, tol=1e-6):
    c = kkt_certificate(prob, sol["x"], sol["s"], sol["y"], sol["z"])
    assert c["rx"] <= tol * c["scale"], c
    assert c["ry"] <= tol * c["scale"], c
    assert c["rz"] <= tol * c["scale"], c
    assert c["s_margin"] >= -1e-9 and c["z_margin"] >= -1e-9, c
    assert abs(c["gap"]) <= tol * (1.0 + abs(c["pobj"])), c
    return c
