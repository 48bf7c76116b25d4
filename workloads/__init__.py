"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package holds only input generation: sparse operators in CSR form and
right-hand sides.  It contains none of the sketched-Krylov arithmetic, so both
the oracle and the CUDA path may consume its outputs without sharing method code.
"""
from .operators import (convdiff_2d, convdiff_3d, upwind_2d, ninepoint_2d, powerlaw_graph_operator,
                        gaussian_rhs, csr_to_scipy, CSR)
from .configs import WORKLOADS, SEEDS, workload

__all__ = ["convdiff_2d", "convdiff_3d", "upwind_2d", "ninepoint_2d", "powerlaw_graph_operator",
           "gaussian_rhs", "csr_to_scipy", "CSR", "WORKLOADS", "SEEDS", "workload"]
