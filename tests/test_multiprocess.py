"""The N-process launch path of bench.py on CPU (gloo, world size 2, 127.0.0.1):
the max-over-ranks reduction used for the timed region, and a torchrun launch of the
reference arm in which rank 0 alone measures and prints one JSON line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    try:
        out.put((rank, bench.reduce_max(10.0 + 5.0 * rank)))
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 15.0), (1, 15.0)]


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--stages", "40"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0


# ---- one batch split over the ranks (paper_2603_29197_gb300/shard.py) ------------------
def test_partition_balances_contiguous_ranges():
    from paper_2603_29197_gb300.shard import partition
    rng = np.random.default_rng(0)
    costs = rng.uniform(10, 60, size=4096) ** 3
    for ws in (1, 2, 3, 4, 8):
        st = partition(costs, ws)
        assert st[0] == 0 and st[-1] == len(costs) and all(a < b for a, b in zip(st, st[1:]))
        shares = np.array([costs[a:b].sum() for a, b in zip(st, st[1:])]) / costs.sum()
        assert np.all(np.abs(shares - 1.0 / ws) <= costs.max() / costs.sum()), (ws, shares)
    assert partition([5.0, 1.0], 4) == [0, 1, 2, 2, 2]      # more ranks than instances
    assert partition([], 2) == [0, 0, 0]


def _oracle_solve(probs, **settings):
    """Stand-in for the GPU batched solve (CPU test): the oracle, instance by instance."""
    from oracle import ipm
    out = []
    for pr in probs:
        r = ipm.solve(pr)
        out.append(dict(status=0 if r.status == "solved" else 2, iters=r.iters, pobj=r.pobj, dobj=r.dobj,
                        x=r.x, y=r.y, z=r.z, s=r.s))
    return 0, out


def _failing_on_rank1(probs, **settings):
    import torch.distributed as dist
    if dist.get_rank() == 1:
        raise RuntimeError("device lost")
    return _oracle_solve(probs)


def _shard_worker(rank, port, out, failing):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2603_29197_gb300.shard import solve_sharded
    from workloads import mpc_batch
    import test_multiprocess as tm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    try:
        probs = mpc_batch(count=10, tmin=10, tmax=40, seed=5)
        res = solve_sharded(probs, solve_fn=tm._failing_on_rank1 if failing else tm._oracle_solve)
        if rank == 0:
            out.put(("ok", [None if r.get("status") is None else (r["status"], r["pobj"]) for r in res["results"]],
                     res["starts"], res["errors"]))
        else:
            out.put(("rank1", res))
    finally:
        dist.destroy_process_group()


def _run_shard(failing):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, port, q, failing)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = [q.get(timeout=10) for _ in range(2)]
    return [g for g in got if g[0] == "ok"][0], [g for g in got if g[0] == "rank1"][0]


def test_sharded_batch_gathers_every_instance_on_rank0():
    """Two gloo ranks split 10 MPC instances by N_K³ into contiguous ranges, solve their
    own ranges and gather status and objective of every instance to rank 0, in the
    original order and equal to a single-process run; rank 1 returns None."""
    from paper_2603_29197_gb300.shard import solve_sharded
    from workloads import mpc_batch
    (_, got, starts, errors), (_, r1) = _run_shard(False)
    assert r1 is None and not errors
    assert 0 < starts[1] < 10
    single = solve_sharded(mpc_batch(count=10, tmin=10, tmax=40, seed=5), solve_fn=_oracle_solve)
    want = [(r["status"], r["pobj"]) for r in single["results"]]
    assert got == want


def test_sharded_batch_reports_a_failing_rank_without_hanging():
    """A rank whose solve raises still joins the gather: rank 0 receives its instances as
    failed (status None) with the error text, and the other rank's results intact."""
    (_, got, starts, errors), _ = _run_shard(True)
    assert set(errors) == {1} and "device lost" in errors[1]
    assert all(g is not None for g in got[:starts[1]])
    assert all(g is None for g in got[starts[1]:])
