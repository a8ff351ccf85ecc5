"""Comparison helper of the GPU parity tests."""
import numpy as np


def rel(a, b):
    """Error of a against the reference b: the larger of the relative l2
    difference ||a - b||_2 / ||b||_2 and max|a - b| / (10 max|b|).

    A value below tol bounds the l2 error by tol and every cell's error by
    10 tol max|b|, so an error confined to a few cells (the ragged edge lane of
    a grid, one inflow row) cannot hide in the norm of the whole field."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.max(np.abs(a))) if a.size else 0.0
    l2 = np.linalg.norm(a - b) / nb
    mc = np.max(np.abs(a - b)) / (10.0 * np.max(np.abs(b)))
    return float(max(l2, mc))
