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
