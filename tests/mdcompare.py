"""Exact comparison helpers for md arrays (test-side only)."""
import math

import numpy as np


def md_diff(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Correctly rounded exact difference of two md arrays [P][K][...] -> [P][...]."""
    P, K = a.shape[:2]
    rest = a.shape[2:]
    A = a.reshape(P, K, -1)
    B = b.reshape(P, K, -1)
    out = np.zeros((P, A.shape[2]))
    for p in range(P):
        for c in range(A.shape[2]):
            out[p, c] = math.fsum(list(A[p, :, c]) + [-v for v in B[p, :, c]])
    return out.reshape((P,) + rest)


def md_value(a: np.ndarray) -> np.ndarray:
    """Correctly rounded double value of an md array [P][K][...] -> [P][...]."""
    P, K = a.shape[:2]
    rest = a.shape[2:]
    A = a.reshape(P, K, -1)
    out = np.zeros((P, A.shape[2]))
    for p in range(P):
        for c in range(A.shape[2]):
            out[p, c] = math.fsum(A[p, :, c])
    return out.reshape((P,) + rest)


def modulus(v: np.ndarray) -> np.ndarray:
    """|.| over planes of a [P][...] double array."""
    return np.sqrt((v ** 2).sum(axis=0))
