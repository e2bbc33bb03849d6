"""The batch analysis assembled from its distinct instance patterns (stack_analysis.cpp)
equals, array for array, the analysis of the whole block-diagonal stack with the
instances' orderings concatenated: KKT rows, columns, value sources, initial values,
diagonal and −W² slots; the ordering, supernodes, row structures, front and update
offsets, relative indices, children, levels, assembly map and pivot signs.  Checked by a
small C++ program (tests/stack_equivalence.cpp) built from the library's host sources,
with AMD and ND, on repeated MPC patterns mixed with other models and edge layouts."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from workloads import Problem, dense_qp, mpc_batch, portfolio_socp, trajectory_socp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_29197_gb300", "csrc")


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("stackeq") / "stack_equivalence")
    srcs = [os.path.join(ROOT, "tests", "stack_equivalence.cpp")] + [
        os.path.join(CSRC, f) for f in ("ordering.cpp", "symbolic.cpp", "kkt_pattern.cpp", "stack_analysis.cpp")]
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), *srcs,
                    "-o", out, "-lpthread"], check=True, capture_output=True)
    return out


def _write(probs, path):
    with open(path, "wb") as f:
        np.array([len(probs)], np.int32).tofile(f)
        for pr in probs:
            np.array([pr.n, pr.m, pr.p, pr.l, len(pr.q)] + list(pr.q), np.int32).tofile(f)
            P = pr.P if pr.P is not None and pr.P.nnz else None
            for M, rows in ((P, pr.n), (pr.A if pr.p else None, pr.p), (pr.G, pr.m)):
                M = sp.csc_matrix((rows, pr.n)) if M is None else sp.csc_matrix(M)
                M.sort_indices()
                np.array([rows, pr.n, M.nnz], np.int32).tofile(f)
                M.indptr.astype(np.int32).tofile(f)
                M.indices.astype(np.int32).tofile(f)
                M.data.astype(np.float64).tofile(f)


def _edge(rng, n, p, l, q, with_P=True):
    m = l + sum(q)
    G = sp.csc_matrix(rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.6))
    P = sp.csc_matrix(np.triu(np.eye(n) * 2.0 + 0.1)) if with_P else sp.csc_matrix((n, n))
    A = sp.csc_matrix(rng.standard_normal((p, n))) if p else sp.csc_matrix((0, n))
    return Problem(n=n, m=m, p=p, P=P, c=rng.standard_normal(n), A=A, b=np.ones(p), G=G, h=np.ones(m), l=l,
                   q=list(q))


BATCHES = {
    "mpc_mixed": lambda: (mpc_batch(count=60, tmin=10, tmax=16, seed=5)[:30]
                          + [dense_qp(n=40, p=8, m=60, rank=6, density=0.1, seed=22),
                             portfolio_socp(n=50, k=6, seed=23), trajectory_socp(N=30, seed=6)]
                          + mpc_batch(count=60, tmin=10, tmax=16, seed=5)[30:]),
    "edge_layouts": lambda: [_edge(np.random.default_rng(7 + r), *k) for r in range(3)
                             for k in ((6, 0, 3, [3]), (5, 2, 0, [3, 2]), (4, 1, 4, [], False), (7, 0, 0, [4, 3]))],
    "mpc_1024": lambda: mpc_batch(count=1024, tmin=10, tmax=60, seed=8),
}


@pytest.mark.parametrize("name", list(BATCHES))
@pytest.mark.parametrize("order", [1, 2])
def test_stacked_analysis_equals_the_whole_stack(prog, tmp_path, name, order):
    path = str(tmp_path / f"{name}.bin")
    _write(BATCHES[name](), path)
    r = subprocess.run([prog, path, str(order)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), (r.stdout[-2000:], r.stderr[-2000:])


def test_comparison_catches_a_planted_difference(prog, tmp_path):
    path = str(tmp_path / "mpc.bin")
    _write(mpc_batch(count=12, tmin=10, tmax=14, seed=9), path)
    r = subprocess.run([prog, path, "2", "plant"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 1 and "FAIL amap_slot" in r.stdout, r.stdout
