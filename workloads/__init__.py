"""Seeded synthetic problem generators shared by the oracle, the tests and the bench.

This package builds problem *data* only (matrices, vectors, cone sizes).  It holds
none of the interior-point method's arithmetic, so that the CPU oracle and the CUDA
path can both draw their inputs from it without sharing any of the method.
"""
from .generators import (  # noqa: F401
    Problem,
    dense_qp,
    trajectory_socp,
    lasso_qp,
    portfolio_socp,
    mpc_batch,
    mpc_instance,
    random_cone_iterate,
)
