"""Pins of the oracle's Newton step on power series (Sections 3 and 4).

* the circle example of Section 3 (printed double-precision digits, and the
  exact Taylor coefficients of cos t in multiple doubles);
* x^2 - 1 - t = 0: x(t) = sqrt(1 + t), coefficients binom(1/2, k);
* (M0 + M1 t) x = c: closed form x(t) = sum_k (-M0^-1 M1)^k M0^-1 c t^k after one step;
* exact-rational brute force of a whole step on tiny random systems;
* backward error of the block Toeplitz solve, degree by degree;
* doubling of the number of correct coefficients per step;
* agreement with the same computation in twice the number of limbs;
* threaded run (one job per polynomial / per right-hand side) bit-identical to serial.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import mdgen
import oracle
from oracle import exact

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def eps(K):
    return Fraction(1, 1 << (52 * K))


def val(x, j, k):
    return exact.md_exact(x, j, k)


def test_circle_double_printed(orc):
    """Section 3, K = 1 (double): the printed digits of x(t)."""
    printed = {}
    with open(os.path.join(GOLD, "circle_double.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, c = line.split()
            printed[int(k)] = float(c)
    s = mdgen.circle_system(1, 8)
    x, norms = orc.newton(s, 5)
    for k in range(9):
        got = float(x[0, 0, 0, k])
        want = printed.get(k, 0.0)
        assert abs(got - want) <= 1e-12 * max(abs(want), 1e-300) + 1e-15, (k, got, want)
    assert norms[-1][1] < 1e-15


@pytest.mark.parametrize("K", [2, 4, 8])
def test_circle_md_exact_cos(orc, K):
    """x(t) = cos t through t^8 exactly: (-1)^j / (2j)!, odd coefficients 0."""
    s = mdgen.circle_system(K, 8)
    x, norms = orc.newton(s, 5)
    for k in range(9):
        want = Fraction((-1) ** (k // 2), __import__("math").factorial(k)) if k % 2 == 0 else Fraction(0)
        got = val(x, 0, k)[0]
        assert abs(got - want) <= 1000 * eps(K), (K, k, float(got - want))


@pytest.mark.parametrize("K,cplx", [(1, False), (2, False), (4, True), (8, False), (10, False)])
def test_sqrt_one_plus_t(orc, K, cplx):
    d = 16
    s = mdgen.sqrt_system(K, d, cplx)
    x, norms = orc.newton(s, 6)
    tol = 1e-13 if K == 1 else None
    for k in range(d + 1):
        want = mdgen.binom_half(k)
        got = val(x, 0, k)
        if K == 1:
            assert abs(float(got[0] - want)) <= tol * max(abs(float(want)), 1e-300) + 1e-16
        else:
            assert abs(got[0] - want) <= 1000 * eps(K) * abs(want), (K, k)
        assert got[1] == 0


@pytest.mark.parametrize("K,cplx", [(2, True), (4, False)])
def test_linear_closed_form(orc, K, cplx):
    n, d = 3, 6
    s, M0, M1, c = mdgen.linear_system(3, n, K, d, cplx)
    x, norms = orc.newton(s, 1)
    # closed form with exact Gaussian elimination
    zero = exact.ZERO
    y = exact.solve_dense(M0, c)  # M0^-1 c
    coeffs = [y]
    for k in range(1, d + 1):
        prev = coeffs[-1]
        v = [zero] * n
        for i in range(n):
            for j in range(n):
                v[i] = exact.cadd(v[i], exact.cmul(M1[i][j], prev[j]))
        w = exact.solve_dense(M0, v)
        coeffs.append([(-a[0], -a[1]) for a in w])
    for k in range(d + 1):
        for j in range(n):
            got = val(x, j, k)
            want = coeffs[k][j]
            scale = max(Fraction(1), abs(want[0]) + abs(want[1]))
            assert abs(got[0] - want[0]) <= 1000 * eps(K) * scale * (k + 1)
            assert abs(got[1] - want[1]) <= 1000 * eps(K) * scale * (k + 1)


@pytest.mark.parametrize("seed,n,d,K", [(1, 2, 4, 2), (2, 3, 3, 2), (3, 2, 5, 3), (4, 3, 2, 4)])
def test_step_exact_brute_force(orc, seed, n, d, K):
    """Whole step against exact rationals (naive AD + dense block Toeplitz elimination)."""
    s = mdgen.random_system(seed, n=n, K=K, cplx=True, d=d, monos=3, maxvars=2, maxdeg=3)
    rng = np.random.default_rng(seed)
    x = s.x0.copy()
    x[:, 0, :, 1:] = rng.uniform(-0.5, 0.5, size=x[:, 0, :, 1:].shape)
    xn, _ = orc.newton_step(s, x)
    xe, dxe, fe, Ae = exact.newton_step_exact(s, x)
    f, A = orc.eval_diff(s, x)
    for i in range(n):
        for k in range(d + 1):
            a, b = val(f, i, k), fe[i][k]
            sc = 1 + abs(b[0]) + abs(b[1])
            assert abs(a[0] - b[0]) <= 1000 * eps(K) * sc * 50 and abs(a[1] - b[1]) <= 1000 * eps(K) * sc * 50
    for j in range(n):
        for k in range(d + 1):
            a, b = val(xn, j, k), xe[j][k]
            sc = 1 + abs(b[0]) + abs(b[1])
            assert abs(a[0] - b[0]) <= 1000 * eps(K) * sc * 100, (j, k, float(a[0] - b[0]))
            assert abs(a[1] - b[1]) <= 1000 * eps(K) * sc * 100


def test_linsolve_backward_error(orc):
    """Per degree: ||b_k - sum_{i<=k} A_i dx_{k-i}|| <= 1e3 eps (sum ||A_i|| ||dx_{k-i}|| + ||b_k||)."""
    K, n, d = 4, 6, 6
    rng = np.random.default_rng(11)
    A = rng.standard_normal((2, K, d + 1, n, n)) * np.array([1.0] + [2.0 ** (-53 * l) for l in range(1, K)])[None, :, None, None, None]
    for k in range(d + 1):
        for c in range(n):
            A[0, 0, k, c, c] += 4.0 if k == 0 else 0.0
    b = rng.standard_normal((2, K, n, d + 1)) * np.array([1.0] + [2.0 ** (-53 * l) for l in range(1, K)])[None, :, None, None]
    # canonicalise limbs exactly
    for arr in (A, b):
        flat = arr.reshape(2, K, -1)
        for p in range(2):
            for c in range(flat.shape[2]):
                flat[p, :, c] = mdgen.md_from_fraction(mdgen.md_to_fraction(flat[p, :, c]), K)
    dx = orc.linsolve(K, True, A, b)
    Ae = exact.mat_series_exact(A)
    be = exact.vec_series_exact(b)
    dxe = exact.vec_series_exact(dx)

    def nrm(v):
        return max(abs(a[0]) + abs(a[1]) for a in v)

    def mnrm(M):
        return max(sum(abs(a[0]) + abs(a[1]) for a in row) for row in M)

    for k in range(d + 1):
        res = list(be[k])
        scale = nrm(be[k])
        for i in range(k + 1):
            for r in range(n):
                for c in range(n):
                    res[r] = exact.csub(res[r], exact.cmul(Ae[i][r][c], dxe[k - i][c]))
            scale += mnrm(Ae[i]) * nrm(dxe[k - i])
        assert nrm(res) <= 1000 * eps(K) * scale, (k, float(nrm(res) / scale))


def test_doubling_of_correct_coefficients(orc):
    """After step s from an exact x0, the residual coefficients 0..2^s - 1 vanish."""
    s = mdgen.config_system(0, seed=3)
    K = s.limbs
    x = s.x0.copy()
    for step in range(1, 5):
        x, _ = orc.newton_step(s, x)
        f, _ = orc.eval_diff(s, x)
        upto = min(s.degree, 2 ** step - 1)
        for i in range(s.n):
            for k in range(upto + 1):
                a = val(f, i, k)
                assert abs(a[0]) + abs(a[1]) <= 1e6 * eps(K), (step, i, k, float(abs(a[0]) + abs(a[1])))
        if 2 ** step <= s.degree:
            big = max(float(abs(val(f, i, 2 ** step)[0]) + abs(val(f, i, 2 ** step)[1])) for i in range(s.n))
            assert big > 1e-20  # not converged yet at that degree


def test_twice_the_limbs(orc):
    """cfg0-type system in dd against the same exact inputs in qd (4 steps)."""
    s2 = mdgen.config_system(0, seed=1)
    s4 = s2.with_limbs(4)
    x2, _ = orc.newton(s2, 4)
    x4, _ = orc.newton(s4, 4)
    for j in range(s2.n):
        for k in range(s2.degree + 1):
            a, b = val(x2, j, k), val(x4, j, k)
            sc = 1 + abs(b[0]) + abs(b[1])
            assert abs(a[0] - b[0]) <= 1000 * eps(2) * sc and abs(a[1] - b[1]) <= 1000 * eps(2) * sc


def test_threads_bit_identical():
    s = mdgen.config_system(0, seed=2)
    o1 = oracle.Oracle(threads=1)
    x1, n1 = o1.newton_step(s, s.x0)
    o4 = oracle.Oracle(threads=4)
    x4, n4 = o4.newton_step(s, s.x0)
    assert np.array_equal(x1, x4) and n1 == n4


def test_singular_a0_reported(orc):
    """A_0 = 0 (all monomials vanish to first order at x0) -> singular."""
    F = Fraction
    polys = [[[(0, 2)], [(1, 1)]]]
    s = mdgen._pack(1, 2, False, 4, polys, [[(F(1), F(0)), (F(1), F(0))]], [(F(0), F(0))], [(F(0), F(0))])
    with pytest.raises(oracle.OracleError, match="singular"):
        orc.newton_step(s, s.x0)
