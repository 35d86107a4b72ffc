"""Parity measures shared by the GPU tests (no GPU needed to import).

An iterate of the CUDA path agrees with the oracle's when both measures stay below the bar:
normwise, ||a - b|| / max(1, ||b||), and element by element, max_i |a_i - b_i| / max(1, ||b||_inf),
so that a few coordinates far off cannot hide inside a large norm.
"""
import numpy as np


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(1.0, np.linalg.norm(b)))


def elem(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


def close(a, b):
    """The larger of the two measures."""
    return max(rel(a, b), elem(a, b))
