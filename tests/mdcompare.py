"""Exact comparison helpers for md arrays (test-side only).

The tolerance of a reduced result (a solve, a Newton step) is read per series
coefficient and per degree: the difference to the reference, divided by the
largest modulus of the reference's coefficients of that degree, must stay
within ``TOL`` unit roundoffs eps_K = 2^(-52 K).
"""
import math

import numpy as np

TOL = 1e3  # unit roundoffs: 1e3 eps_K per degree


def eps(K: int) -> float:
    """Unit roundoff of K-limb arithmetic, 2^(-52 K)."""
    return 2.0 ** (-52 * K)


def md_diff(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Correctly rounded exact difference of two md arrays [P][Ka][...] and
    [P][Kb][...] (the limb counts may differ) -> [P][...]."""
    P, Ka = a.shape[:2]
    Kb = b.shape[1]
    rest = a.shape[2:]
    assert b.shape[0] == P and b.shape[2:] == rest, (a.shape, b.shape)
    A = a.reshape(P, Ka, -1)
    B = b.reshape(P, Kb, -1)
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


def rel_by_degree(got: np.ndarray, want: np.ndarray) -> np.ndarray:
    """Series [P][K][n][d+1]: max over unknowns of |got - want| divided by the
    largest |want| of the same degree, one value per degree k."""
    diff = modulus(md_diff(got, want))  # [n][d+1]
    scale = np.maximum(modulus(md_value(want)).max(axis=0), 1e-300)
    return diff.max(axis=0) / scale


def worst_in_eps(got: np.ndarray, want: np.ndarray, K: int) -> float:
    """Largest per-degree relative difference in units of eps_K."""
    return float((rel_by_degree(got, want) / eps(K)).max())
