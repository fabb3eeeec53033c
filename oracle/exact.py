"""Exact-rational brute force for tiny systems (test infrastructure only).

Independent of both the C oracle and the CUDA path, and deliberately a
different algorithm:

* monomials are expanded naively (powers by repeated series products) and
  differentiated by the exponent rule, with no Speelpenning products and no
  common factor;
* the linearized system A(t) dx(t) = -f(t) of Section 4 is assembled as the
  dense (d+1)n x (d+1)n lower triangular block Toeplitz matrix and solved by
  Gaussian elimination over the Gaussian rationals;
* for N > n equations, each degree's least squares problem is solved through
  its normal equations over the Gaussian rationals.

All arithmetic is exact (``fractions.Fraction``); inputs are the exact values
of the md limbs.
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Tuple

import numpy as np

C = Tuple[Fraction, Fraction]
ZERO: C = (Fraction(0), Fraction(0))
ONE: C = (Fraction(1), Fraction(0))


def cadd(a: C, b: C) -> C:
    return (a[0] + b[0], a[1] + b[1])


def csub(a: C, b: C) -> C:
    return (a[0] - b[0], a[1] - b[1])


def cmul(a: C, b: C) -> C:
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def cdiv(a: C, b: C) -> C:
    den = b[0] * b[0] + b[1] * b[1]
    return ((a[0] * b[0] + a[1] * b[1]) / den, (a[1] * b[0] - a[0] * b[1]) / den)


def cabs2(a: C) -> Fraction:
    return a[0] * a[0] + a[1] * a[1]


def md_exact(arr: np.ndarray, *index) -> C:
    """Exact value of the md number at [p][:][index...] of a [P][K][...] array."""
    P = arr.shape[0]
    re = sum((Fraction(float(v)) for v in arr[(0, slice(None)) + tuple(index)]), Fraction(0))
    im = sum((Fraction(float(v)) for v in arr[(1, slice(None)) + tuple(index)]), Fraction(0)) if P == 2 else Fraction(0)
    return (re, im)


def series_mul(x: List[C], y: List[C], d: int) -> List[C]:
    z = [ZERO] * (d + 1)
    for i in range(d + 1):
        if x[i] == ZERO:
            continue
        for j in range(d + 1 - i):
            z[i + j] = cadd(z[i + j], cmul(x[i], y[j]))
    return z


def series_pow(x: List[C], e: int, d: int) -> List[C]:
    r = [ONE] + [ZERO] * d
    for _ in range(e):
        r = series_mul(r, x, d)
    return r


def eval_diff_exact(s, x: np.ndarray):
    """Exact f (list over the N polynomials of series) and A (list over k of
    N x n lists) at the series x."""
    n, d = s.n, s.degree
    N = getattr(s, "N", n)
    xs = [[md_exact(x, j, k) for k in range(d + 1)] for j in range(n)]
    tser = [ZERO, ONE] + [ZERO] * (d - 1) if d >= 1 else [ZERO]
    allv = xs + [tser]
    f = []
    A = [[[ZERO] * n for _ in range(N)] for _ in range(d + 1)]
    for i in range(N):
        fi = [md_exact(s.cst, i)] + [ZERO] * d
        for m, pairs in s.monomials(i):
            c = md_exact(s.coef, m)
            powers = {v: series_pow(allv[v], e, d) for v, e in pairs}
            val = [c] + [ZERO] * d
            for v, _ in pairs:
                val = series_mul(val, powers[v], d)
            fi = [cadd(a, b) for a, b in zip(fi, val)]
            for v, e in pairs:
                if v == n:
                    continue
                der = [cmul(c, (Fraction(e), Fraction(0)))] + [ZERO] * d
                der = series_mul(der, series_pow(allv[v], e - 1, d), d)
                for v2, _ in pairs:
                    if v2 != v:
                        der = series_mul(der, powers[v2], d)
                for k in range(d + 1):
                    A[k][i][v] = cadd(A[k][i][v], der[k])
        f.append(fi)
    return f, A


def solve_dense(M: List[List[C]], rhs: List[C]) -> List[C]:
    """Gaussian elimination over Q(i) (exact; first nonzero pivot)."""
    N = len(rhs)
    M = [row[:] for row in M]
    rhs = rhs[:]
    for c in range(N):
        piv = next(r for r in range(c, N) if M[r][c] != ZERO)
        if piv != c:
            M[c], M[piv] = M[piv], M[c]
            rhs[c], rhs[piv] = rhs[piv], rhs[c]
        inv = cdiv(ONE, M[c][c])
        for r in range(c + 1, N):
            if M[r][c] == ZERO:
                continue
            fct = cmul(M[r][c], inv)
            for cc in range(c, N):
                M[r][cc] = csub(M[r][cc], cmul(fct, M[c][cc]))
            rhs[r] = csub(rhs[r], cmul(fct, rhs[c]))
    x = [ZERO] * N
    for r in range(N - 1, -1, -1):
        acc = rhs[r]
        for cc in range(r + 1, N):
            acc = csub(acc, cmul(M[r][cc], x[cc]))
        x[r] = cdiv(acc, M[r][r])
    return x


def block_toeplitz_solve(A: List[List[List[C]]], b: List[List[C]]) -> List[List[C]]:
    """A[k] n x n (row-major lists), b[k] length n -> dx[k] by one dense solve."""
    D1 = len(A)
    n = len(b[0])
    N = D1 * n
    M = [[ZERO] * N for _ in range(N)]
    for bi in range(D1):
        for bj in range(bi + 1):
            blk = A[bi - bj]
            for r in range(n):
                for c in range(n):
                    M[bi * n + r][bj * n + c] = blk[r][c]
    rhs = [b[k][i] for k in range(D1) for i in range(n)]
    sol = solve_dense(M, rhs)
    return [[sol[k * n + i] for i in range(n)] for k in range(D1)]


def block_lstsq(A: List[List[List[C]]], b: List[List[C]]) -> List[List[C]]:
    """Least squares block Toeplitz solve over Q(i), A[k] N x n, b[k] length N:
    per degree dx_k solves the normal equations A_0^H A_0 dx_k = A_0^H r_k,
    r_k = b_k - sum_{j<k} A_{k-j} dx_j (the minimiser of ||A_0 dx_k - r_k||)."""
    D1, N, n = len(A), len(A[0]), len(A[0][0])

    def conj(z):
        return (z[0], -z[1])

    A0 = A[0]
    G = [[ZERO] * n for _ in range(n)]
    for r in range(n):
        for c in range(n):
            acc = ZERO
            for i in range(N):
                acc = cadd(acc, cmul(conj(A0[i][r]), A0[i][c]))
            G[r][c] = acc
    dx = []
    for k in range(D1):
        rk = list(b[k])
        for j in range(k):
            for i in range(N):
                for c in range(n):
                    rk[i] = csub(rk[i], cmul(A[k - j][i][c], dx[j][c]))
        h = [ZERO] * n
        for r in range(n):
            for i in range(N):
                h[r] = cadd(h[r], cmul(conj(A0[i][r]), rk[i]))
        dx.append(solve_dense(G, h))
    return dx


def newton_step_exact(s, x: np.ndarray):
    """Exact step from the md input x: returns (x_new[j][k], dx[k][j], f, A)."""
    n, d = s.n, s.degree
    N = getattr(s, "N", n)
    f, A = eval_diff_exact(s, x)
    b = [[(-f[i][k][0], -f[i][k][1]) for i in range(N)] for k in range(d + 1)]
    dx = block_toeplitz_solve(A, b) if N == n else block_lstsq(A, b)
    xn = [[cadd(md_exact(x, j, k), dx[k][j]) for k in range(d + 1)] for j in range(n)]
    return xn, dx, f, A


def mat_series_exact(A: np.ndarray):
    """[P][K][d+1][n(col)][N(row)] -> A[k][row][col] exact."""
    D1, n, N = A.shape[2], A.shape[3], A.shape[4]
    return [[[md_exact(A, k, c, r) for c in range(n)] for r in range(N)] for k in range(D1)]


def vec_series_exact(b: np.ndarray):
    """[P][K][n][d+1] -> b[k][i] exact."""
    n, D1 = b.shape[2], b.shape[3]
    return [[md_exact(b, i, k) for i in range(n)] for k in range(D1)]
