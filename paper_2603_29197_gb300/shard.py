"""One batch of independent problems split over the ranks of a process group (one GPU
per rank): contiguous instance ranges balanced by the instances' work, a batched solve
per rank (qoco_gpu_setup_batch), and one gather of every instance's result to rank 0.

The instances are independent, so nothing crosses ranks while they are solved; the only
exchange is the final gather of status, iteration count, objectives and solution vectors.
The work of an instance is taken as N_K³ (N_K = n + p + m, its KKT dimension): the
factorisation of a banded or dense KKT block grows at most that fast, and the split only
needs the ranks' shares to be about equal.
"""
from __future__ import annotations

import numpy as np


def instance_cost(prob) -> float:
    """Work estimate of one instance: N_K³."""
    nk = float(prob.n + prob.p + prob.m)
    return nk ** 3


def partition(costs, world_size: int):
    """Contiguous ranges [starts[r], starts[r+1]) of the instances, one per rank, whose
    cost sums are as equal as a prefix split allows: the boundary after rank r − 1 is the
    instance boundary nearest to r/world_size of the total cost, kept strictly increasing
    so that every rank has at least one instance while there are enough of them."""
    costs = np.asarray(costs, dtype=np.float64)
    n = len(costs)
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    if n <= world_size:  # one instance per rank while they last
        return [min(r, n) for r in range(world_size + 1)]
    cum = np.concatenate([[0.0], np.cumsum(costs)])  # cum[k] = cost of instances [0, k)
    total = cum[-1]
    starts = [0]
    for r in range(1, world_size):
        target = total * r / world_size
        k = int(np.searchsorted(cum, target, side="left"))  # first k with cum[k] ≥ target
        if k > 0 and target - cum[k - 1] < cum[min(k, n)] - target:
            k -= 1
        left = world_size - r  # ranks still to fill after this boundary, one instance each
        starts.append(min(max(k, starts[-1] + 1), n - left))
    starts.append(n)
    return starts


def _gpu_solve(probs, **settings):
    """Batched GPU solve of one rank's instances (the default solve function)."""
    from . import BatchSolver
    S = BatchSolver(probs, **settings)
    try:
        status = S.solve()
        info = S.batch_info()
        sols = S.instance_solutions()
    finally:
        S.close()
    return status, [dict(status=int(info["status"][i]), iters=int(info["iters"][i]), pobj=float(info["pobj"][i]),
                         dobj=float(info["dobj"][i]), x=sols[i]["x"], y=sols[i]["y"], z=sols[i]["z"],
                         s=sols[i]["s"]) for i in range(len(probs))]


def solve_sharded(probs, group=None, solve_fn=None, **settings):
    """Solves `probs` (the same list on every rank) split over the ranks of `group` (the
    default process group; a plain batched solve without one).  Returns, on rank 0, the
    per-instance results in the original order and the ranges used; None on the other
    ranks.  A rank whose solve raises still takes part in the gather (its instances are
    reported with status None and the error text), so no rank is left waiting."""
    import torch.distributed as dist
    solve_fn = solve_fn or _gpu_solve
    dist_on = dist.is_available() and dist.is_initialized()
    ws = dist.get_world_size(group) if dist_on else 1
    rank = dist.get_rank(group) if dist_on else 0
    starts = partition([instance_cost(p) for p in probs], ws)
    mine = probs[starts[rank]:starts[rank + 1]]
    err = None
    results = []
    if mine:
        try:
            _, results = solve_fn(mine, **settings)
        except Exception as e:  # reported through the gather
            err = f"{type(e).__name__}: {e}"
            results = [dict(status=None, error=err) for _ in mine]
    payload = (rank, starts[rank], results, err)
    if not dist_on or ws == 1:
        gathered = [payload]
    else:
        gathered = [None] * ws if rank == 0 else None
        dist.gather_object(payload, gathered, dst=0, group=group)
    if rank != 0:
        return None
    out = [None] * len(probs)
    errors = {}
    for r, start, res, e in gathered:
        if e:
            errors[r] = e
        for k, item in enumerate(res):
            out[start + k] = item
    return dict(results=out, starts=starts, errors=errors)
