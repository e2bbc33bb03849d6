"""GPU parity of the cone kernels (NT scaling, Jordan product and division, max
step) against the oracle at shared random iterates, through the C ABI."""
import math

import numpy as np
import pytest

from oracle import cones as oc
from workloads import random_cone_iterate

from _gpu_util import blockwise_rel

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(2024)
LAYOUTS = [
    (0, [2]), (0, [3]), (5, [4]), (3, [2, 3, 4, 7]), (0, [201]), (7, []), (4, [4] * 6 + [33]),
    # ragged mixes spanning several blocks of the orthant / small / large groups
    (1000, [4] * 700), (257, list(RNG.integers(2, 70, 400))), (0, [32, 33, 64, 500, 2, 1025]),
    (513, [3] * 300 + [40] * 9),
]


def T(a):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda()


def N(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def q():
    import paper_2603_29197_gb300 as qq
    return qq


@pytest.mark.parametrize("l,qs", LAYOUTS)
@pytest.mark.parametrize("spread", [0.0, 4.0])
def test_nt_scaling(q, l, qs, spread):
    s, z, _, _ = random_cone_iterate(l, qs, seed=1 + l + len(qs), scale_spread=spread)
    C = q.Cones(l, qs)
    w, eta, lam = C.nt_scaling(T(s), T(z))
    W = oc.NTScaling(s, z, l, qs)
    w, eta, lam = N(w), N(eta), N(lam)
    if l:
        np.testing.assert_allclose(w[:l], W.w, rtol=1e-14)
    for k, (o, d) in enumerate(oc.blocks(l, qs)):
        np.testing.assert_allclose(w[o:o + d], W.wbar[k], rtol=1e-11, atol=1e-11 * np.abs(W.wbar[k]).max())
        assert math.isclose(eta[k], W.eta[k], rel_tol=1e-12)
    assert blockwise_rel(lam, W.lam, l, qs) <= 1e-11


@pytest.mark.parametrize("l,qs", LAYOUTS)
def test_product_and_division(q, l, qs):
    rng = np.random.default_rng(7)
    m = l + int(sum(qs))
    u, v = rng.standard_normal(m), rng.standard_normal(m)
    C = q.Cones(l, qs)
    got = N(C.product(T(u), T(v)))
    ref = oc.jordan_product(u, v, l, qs)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(ref).max()))
    s, z, _, _ = random_cone_iterate(l, qs, seed=9)
    lam = oc.NTScaling(s, z, l, qs).lam
    got = N(C.division(T(lam), T(v)))
    ref = oc.jordan_division(lam, v, l, qs)
    assert blockwise_rel(got, ref, l, qs) <= 1e-10


@pytest.mark.parametrize("l,qs", LAYOUTS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_max_step(q, l, qs, seed):
    s, _, ds, _ = random_cone_iterate(l, qs, seed=seed)
    C = q.Cones(l, qs)
    got = float(N(C.max_step(T(s), T(ds)))[0])
    ref = oc.max_step(s, ds, l, qs)
    if math.isinf(ref):
        assert math.isinf(got)
    else:
        assert math.isclose(got, ref, rel_tol=1e-10), (got, ref)
    capped = float(N(C.max_step(T(s), T(ds), cap=0.5 * min(ref, 1.0)))[0])
    assert capped == 0.5 * min(ref, 1.0) or math.isclose(capped, 0.5 * min(ref, 1.0), rel_tol=1e-15)


def test_max_step_unbounded_direction(q):
    l, qs = 3, [4, 40]
    s, _, _, _ = random_cone_iterate(l, qs, seed=5)
    C = q.Cones(l, qs)
    # ds = s is inside the cone: no finite step
    got = float(N(C.max_step(T(s), T(s)))[0])
    assert math.isinf(got)
    assert float(N(C.max_step(T(s), T(s), cap=1.0))[0]) == 1.0


def test_max_step_reuses_caller_scratch(q):
    l, qs = 600, [3] * 500
    C = q.Cones(l, qs)
    import torch
    scratch = torch.full((C.max_step_scratch_bytes() // 8 + 1,), float("nan"), dtype=torch.float64,
                         device="cuda")
    for seed in range(3):
        s, _, ds, _ = random_cone_iterate(l, qs, seed=seed)
        got = float(N(C.max_step(T(s), T(ds), scratch=scratch))[0])
        assert math.isclose(got, oc.max_step(s, ds, l, qs), rel_tol=1e-10)
