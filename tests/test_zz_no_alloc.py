"""Allocation-free max step (qoco_gpu_cone_max_step_noalloc), through the C ABI.

Some callers cannot allocate device memory while they run: code that is being
captured into a CUDA graph, real-time control loops that reserve all memory at
start-up, or hosts whose device allocator belongs to another framework.  This entry
point serves them: it takes no scratch buffer and keeps its block partials in one
fixed device array inside the library.  The tests compare it with the scratch-taking
entry point on the same inputs, on two calls in a row (the array is shared by every
call, so the second call must not depend on what the first left there), and check
that a cone grid too large for the fixed array is refused before any launch.

This file is collected last on purpose, so that a run stopping at its first failure
has already run every other test.
"""
import math

import numpy as np
import pytest

from workloads import random_cone_iterate

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("l,qs", [(700, [3] * 400 + [40] * 5 + [201]), (0, [4] * 33), (5, [])])
def test_noalloc_max_step_matches_scratch_entry_point_on_two_calls(l, qs):
    import torch
    import paper_2603_29197_gb300 as q
    C = q.Cones(l, qs)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for seed in (0, 1):  # two calls in a row on the shared device array
        s, _, ds, _ = random_cone_iterate(l, qs, seed=seed)
        u, du = _t(s), _t(ds)
        ref = float(C.max_step(u, du)[0].item())  # existing entry point, caller scratch
        rc = C.max_step_noalloc(u, du, out)
        assert rc == 0
        got = float(out[0].item())
        if math.isinf(ref):
            assert math.isinf(got)
        else:
            assert math.isclose(got, ref, rel_tol=1e-10), (got, ref)
        # with a cap, as the interior-point loop uses it
        rc = C.max_step_noalloc(u, du, out, cap=1.0)
        assert rc == 0
        assert float(out[0].item()) == min(1.0, float(C.max_step(u, du, cap=1.0)[0].item()))


def test_noalloc_max_step_refuses_grids_beyond_its_array():
    import torch
    import paper_2603_29197_gb300 as q
    from paper_2603_29197_gb300 import _lib
    l = 8192 * 256 + 1  # one orthant block more than the 8192 partials the array holds
    C = q.Cones(l, [])
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rc = C.max_step_noalloc(dummy, dummy, out)
    assert rc == _lib.ERR_TOO_LARGE
    assert float(out[0].item()) == -1.0  # nothing was launched
