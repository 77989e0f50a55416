"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def rel_l2(a, b):
    a = np.asarray(a, float).ravel()
    b = np.asarray(b, float).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def need_gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lib_built():
    from paper_1802_05246_b300 import build

    build.build()
    import paper_1802_05246_b300 as hb

    return hb


def hermite_cond(m):
    """Condition number of the (2m+2)x(2m+2) confluent Vandermonde system of
    Eq. (Hermcon) that the oracle solves by LU for every fibre."""
    import math

    n = 2 * m + 2
    A = np.zeros((n, n))
    for s, xi in enumerate((-0.5, 0.5)):
        for l in range(m + 1):
            for j in range(l, n):
                A[s * (m + 1) + l, j] = math.comb(j, l) * xi ** (j - l)
    return float(np.linalg.cond(A))


def run_tol(m, base=1e-11):
    """Parity tolerance for a run against the oracle: base up to m = 4, scaled
    by the growth of the oracle's LU forward error (cond ratio) beyond."""
    return base * max(1.0, hermite_cond(m) / hermite_cond(4))
