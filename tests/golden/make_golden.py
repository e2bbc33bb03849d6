"""Writes the stored expected values for the full-size parity tests: a JSON summary
(status, iterations, objectives, norms, 64 sampled entries per vector) and a compressed
.npz with every entry of x, y, z and s.

Every value comes from the CPU oracle (oracle/ipm.py) run on the seeded generator
instance; nothing here touches the CUDA library.  Usage:

    python tests/golden/make_golden.py trajectory_socp_N20000 [portfolio_socp_n20000 ...]
    python tests/golden/make_golden.py mpc_batch_4096_sample
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ipm  # noqa: E402
from workloads import lasso_qp, mpc_batch, portfolio_socp, trajectory_socp  # noqa: E402

CASES = {
    "trajectory_socp_N20000": lambda: trajectory_socp(N=20000, seed=0),
    "portfolio_socp_n20000": lambda: portfolio_socp(n=20000, k=200, seed=0),
    # the lasso QP scaled by 1/10 per dimension with the same 50 nonzeros per row of F
    "lasso_qp_r5000_c10000": lambda: lasso_qp(rows=5000, cols=10000, density=5e-3, seed=0),
}


def sample_idx(n, k=64, seed=123):
    rng = np.random.default_rng(seed)
    return sorted(set(rng.choice(n, size=min(k, n), replace=False).tolist()))


def make(name):
    prob = CASES[name]()
    t0 = time.time()
    r = ipm.solve(prob)
    dt = time.time() - t0
    out = dict(name=name, status=r.status, iters=r.iters, pobj=r.pobj, dobj=r.dobj,
               oracle_seconds=dt, n=prob.n, m=prob.m, p=prob.p,
               x_inf=float(np.abs(r.x).max()), y_inf=float(np.abs(r.y).max(initial=0.0)),
               z_inf=float(np.abs(r.z).max(initial=0.0)))
    for key, vec in (("x", r.x), ("y", r.y), ("z", r.z), ("s", r.s)):
        if vec.size:
            idx = sample_idx(vec.size)
            out[f"{key}_idx"] = idx
            out[f"{key}_val"] = [float(vec[i]) for i in idx]
    meta = {k: (v.tolist() if isinstance(v, np.ndarray) and v.size < 16 else v)
            for k, v in prob.meta.items() if isinstance(v, (int, float, np.ndarray)) and
            (not isinstance(v, np.ndarray) or v.size < 16)}
    out["generator_meta"] = meta
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    np.savez_compressed(path[:-5] + ".npz", x=r.x, y=r.y, z=r.z, s=r.s)
    print(name, r.status, r.iters, r.pobj, f"{dt:.1f}s")


def make_mpc_sample(name="mpc_batch_4096_sample", count=4096, k=16):
    """Oracle solutions of a seeded sample of the MPC batch (status, iterations, objective)."""
    probs = mpc_batch(count=count, seed=0)
    idx = sorted(np.random.default_rng(7).choice(count, size=k, replace=False).tolist())
    out = dict(name=name, count=count, idx=idx, status=[], iters=[], pobj=[])
    for i in idx:
        r = ipm.solve(probs[i])
        out["status"].append(r.status)
        out["iters"].append(r.iters)
        out["pobj"].append(r.pobj)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, out["status"])


if __name__ == "__main__":
    for nm in sys.argv[1:] or list(CASES) + ["mpc_batch_4096_sample"]:
        if nm == "mpc_batch_4096_sample":
            make_mpc_sample()
        else:
            make(nm)
