"""Structural invariants of the host symbolic analysis, checked by a small C++ program
(tests/host_invariants.cpp) built from the library's host sources: the KKT pattern is
sorted and symmetric with every diagonal; the ordering is a permutation; supernodes are
contiguous and postordered; each front lists its own columns first and its update rows
sorted below them; every lower entry of the permuted matrix falls inside its column's
front and is assembled exactly once at its front position; children's update rows are
rows of the parent at their relative indices; levels grow towards the roots; the launch
plan puts every front in exactly one factor list and one solve list, and its dataflow
items list children strictly before parents (the condition under which the dataflow
kernels' bounded waits always end).  These are the facts the device factorisation and
solves index by."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from workloads import Problem, dense_qp, lasso_qp, mpc_batch, portfolio_socp, trajectory_socp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_29197_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("hostinv") / "host_invariants")
    srcs = [os.path.join(ROOT, "tests", "host_invariants.cpp")] + [
        os.path.join(CSRC, f) for f in ("ordering.cpp", "symbolic.cpp", "kkt_pattern.cpp", "plan.cpp")]
    cmd = ["g++", "-O1", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), *srcs, "-o", out,
           "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


def _write(prob, d):
    os.makedirs(d, exist_ok=True)

    def w(M, name):
        M = sp.csc_matrix(M)
        np.array([M.shape[0], M.shape[1], M.nnz], dtype=np.int32).tofile(os.path.join(d, f"{name}_hdr.bin"))
        M.indptr.astype(np.int32).tofile(os.path.join(d, f"{name}_p.bin"))
        M.indices.astype(np.int32).tofile(os.path.join(d, f"{name}_i.bin"))
        M.data.astype(np.float64).tofile(os.path.join(d, f"{name}_x.bin"))

    P = sp.triu(prob.P).tocsc() if prob.P is not None else sp.csc_matrix((prob.n, prob.n))
    w(P, "P")
    w(prob.A if prob.p else sp.csc_matrix((0, prob.n)), "A")
    w(prob.G, "G")
    np.array([prob.n, prob.m, prob.p, prob.l, len(prob.q)] + list(prob.q), dtype=np.int32).tofile(
        os.path.join(d, "dims.bin"))


def _stack(probs):
    P = sp.block_diag([sp.csc_matrix(p.P) for p in probs], format="csc")
    A = sp.block_diag([sp.csc_matrix(p.A) for p in probs], format="csc")
    G = sp.vstack([sp.block_diag([sp.csc_matrix(p.G)[:p.l] for p in probs]),
                   sp.block_diag([sp.csc_matrix(p.G)[p.l:] for p in probs])]).tocsc()
    return Problem(n=P.shape[0], m=G.shape[0], p=A.shape[0], P=P, c=np.zeros(P.shape[0]), A=A,
                   b=np.zeros(A.shape[0]), G=G, h=np.zeros(G.shape[0]), l=sum(p.l for p in probs),
                   q=sum([list(p.q) for p in probs], []))


CASES = {
    "dense_qp": (lambda: dense_qp(n=120, p=30, m=200, rank=10, density=0.05, seed=2), 1, (0, 1, 2, 3)),
    "trajectory": (lambda: trajectory_socp(N=400, seed=3), 1, (0, 1, 2)),
    "portfolio": (lambda: portfolio_socp(n=600, k=30, seed=4), 1, (0, 1, 2, 3)),
    "lasso": (lambda: lasso_qp(rows=300, cols=600, density=0.02, seed=5), 1, (0, 1, 2)),
    "mpc_stack": (lambda: _stack(mpc_batch(count=40, tmin=10, tmax=60, seed=6)), 40, (0, 1, 2)),
    # levels wide enough (≥ 2432 fronts above one thread's order) for the dataflow
    # factorisation's one-thread batches, warp groups and two-to-a-warp groups
    "trajectory_wide": (lambda: trajectory_socp(N=20000, seed=3), 1, (2,)),
    # a dense Schur complement on the equality rows: thin children with updates of more
    # than 1024 rows are absorbed into the root front (columns re-emitted out of postorder)
    "lasso_absorb": (lambda: lasso_qp(rows=5000, cols=10000, density=1e-2, seed=0), 1, (1,)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_symbolic_analysis_invariants(checker, tmp_path, name):
    make, trees, orders = CASES[name]
    d = str(tmp_path / name)
    _write(make(), d)
    for order in orders:
        r = subprocess.run([checker, d, str(order), str(trees)], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, (order, r.stdout[-2000:], r.stderr[-2000:])
        assert r.stdout.startswith("ok"), r.stdout
        if name == "mpc_stack":  # all fronts fit a warp: both dataflow plans were checked
            assert "solve 1 factor 1" in r.stdout, r.stdout
        if name == "trajectory_wide":  # every kind of dataflow factorisation item occurs
            items = [int(v) for v in r.stdout.split("items")[1].split()[:4]]
            assert "factor 1" in r.stdout and min(items) > 0, r.stdout


@pytest.mark.parametrize("plant", ["plant_rel", "plant_map"])
def test_checker_catches_a_planted_error(checker, tmp_path, plant):
    d = str(tmp_path / "traj")
    _write(trajectory_socp(N=200, seed=7), d)
    r = subprocess.run([checker, d, "2", "1", plant], capture_output=True, text=True, timeout=300)
    assert r.returncode == 1 and "FAIL" in r.stdout, r.stdout


def test_thin_children_with_large_updates_are_absorbed_into_the_root():
    """The scaled lasso's Schur complement on its 5000 equality rows is dense: its root
    front has thin children (a few columns each) whose updates span 2500–4000 of the
    root's rows.  After the absorption pass no front but the root has more than 1024
    rows and the front storage is the root's plus small fronts."""
    import paper_2603_29197_gb300 as q
    prob = lasso_qp(rows=5000, cols=10000, density=1e-2, seed=0)
    info, perm, sn, fs, lv = q.analyze(prob, structure=True, ordering=1)
    big = np.sort(fs)[::-1]
    assert big[0] >= 5000 and big[1] < 1024, big[:4]
    # front storage: the root's f² plus small fronts (the separate children took 81e6 more)
    assert info["front_entries"] < big[0] ** 2 + 30e6, info["front_entries"]
