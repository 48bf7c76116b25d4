"""Shared helpers of the GPU parity tests: upload a workload, run the oracle."""
import math

import numpy as np
import torch

from workloads import csr_to_scipy, gaussian_rhs


def upload(skf, A):
    return skf.upload_csr(A.rowptr, A.colind, A.values, device="cuda")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rhs(N, seed=12):
    b = gaussian_rhs(N, seed)
    return b, torch.as_tensor(b, device="cuda")
