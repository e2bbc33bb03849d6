"""CPU oracle for the QOCO-style interior-point hot path — TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of what the GPU path computes, written from the
paper (QOCO-GPU, §1 eq. (1), §2 eq. (2), §2.3) and from the standard Nesterov–Todd /
Mehrotra mathematics that the paper defers to (its refs. to QOCO and to the CVXOPT
notes).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product package never does, and this package never
imports the product package.

Modules
  cones  — Jordan algebra, NT scaling, max step, projection, shift into the cone
  kkt    — KKT assembly (eq. (2) with static regularisation), solve + refinement,
           a dense LDLᵀ for tiny cases
  ipm    — the predictor–corrector loop

Parity status: every function here is pinned by tests/test_oracle_*.py against
closed forms, identities, brute force or textbook special cases (see each
module's header); none is "parity unpinned".
"""
