"""Helpers shared by the GPU tests (marked ``gpu``)."""
import numpy as np
import pytest


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    return torch


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def db_err(a, b):
    return float(np.max(np.abs(20 * np.log10(np.abs(a) / np.abs(b)))))
