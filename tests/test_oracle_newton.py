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
import copy
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


@pytest.mark.parametrize("method", [0, 1])
def test_linsolve_backward_error(orc, method):
    """Per degree: ||b_k - sum_{i<=k} A_i dx_{k-i}|| <= 1e3 eps (sum ||A_i|| ||dx_{k-i}|| + ||b_k||);
    A_0 factored by Householder QR (method 0) or LU with partial pivoting (1)."""
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
    dx = orc.linsolve(K, True, A, b, method=method)
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


# ------------------------------------------- Newton with degree continuation
def _sqrt_start(K, D):
    """x^2 - 1 - t = 0 from x0 = 1 + t/2 (coefficients 0 and 1 exact)."""
    s = mdgen.sqrt_system(K, D)
    x0 = s.x0.copy()
    x0[0, 0, 0, 1] = 0.5
    return s, x0


def _exact_sqrt_newton(d, steps):
    """Exact rational Newton on x^2 - 1 - t from 1 + t/2, truncated at degree d:
    returns the list of updates dx (coefficient lists) of every step."""
    F = Fraction
    x = [F(1), F(1, 2)] + [F(0)] * (d - 1)
    out = []
    for _ in range(steps):
        f = [sum(x[i] * x[k - i] for i in range(k + 1)) for k in range(d + 1)]
        f[0] -= 1
        f[1] -= 1
        a = [2 * v for v in x]  # A(t) = 2 x(t); dx = -f / a as a series division
        dx = []
        for k in range(d + 1):
            dx.append((-f[k] - sum(a[k - i] * dx[i] for i in range(k))) / a[0])
        x = [u + v for u, v in zip(x, dx)]
        out.append(dx)
    return out


@pytest.mark.parametrize("K,tol", [(2, 1e-28), (4, 1e-58)])
def test_newton_run_doubling_pins_iterations(orc, K, tol):
    """Newton on series doubles the number of correct coefficients per step.
    From 2 correct coefficients, degree 8 (9 coefficients) is exact after 3
    steps, so the 4th step's update is rounding-sized: 4 steps.  Degree 16
    then starts with 9 correct coefficients, one step makes 18: 2 steps."""
    s, x0 = _sqrt_start(K, 16)
    x, rep = orc.newton_run(s, [8, 16], [8, 8], tol, 1.0, x0)
    assert rep["levels_done"] == 2 and rep["converged"]
    assert rep["iterations"] == [4, 2]
    for k in range(17):
        want = mdgen.binom_half(k)
        got = val(x, 0, k)
        assert abs(got[0] - want) <= 1000 * eps(K) * abs(want), (k, float(got[0] - want))


def test_newton_run_too_large_stops_ladder(orc):
    """Two steps at degree 8 leave coefficient 8 wrong: the last update equals
    the exact rational one, it is above too_large, and degree 16 is not run."""
    s, x0 = _sqrt_start(2, 16)
    x, rep = orc.newton_run(s, [8, 16], [2, 8], 1e-28, 1e-6, x0)
    assert rep["levels_done"] == 1 and not rep["converged"] and rep["iterations"] == [2]
    dx = _exact_sqrt_newton(8, 2)
    assert rep["dx_norm"][0] == pytest.approx(abs(float(dx[1][8])), rel=1e-15)
    assert rep["dx_max"][0] == pytest.approx(max(abs(float(v)) for v in dx[1]), rel=1e-15)
    # coefficients above degree 8 were not touched
    assert np.all(x[..., 9:] == x0[..., 9:])
    # the same ladder with a larger threshold goes on to degree 16
    _, rep2 = orc.newton_run(s, [8, 16], [2, 8], 1e-28, 1.0, x0)
    assert rep2["levels_done"] == 2 and rep2["iterations"][0] == 2


def test_newton_run_equals_repeated_steps(orc):
    """A one-level ladder is the plain step repeated; the level's series then
    continues the next level (cfg0-type dd complex system)."""
    s = mdgen.config_system(0, seed=4)
    x_run, rep = orc.newton_run(s, [s.degree], [3], 0.0, 1e300)
    x = s.x0.copy()
    for _ in range(3):
        x, nr = orc.newton_step(s, x)
    assert rep["iterations"] == [3] and np.array_equal(x_run, x)
    assert rep["dx_norm"][0] == nr[0] and rep["dx_max"][0] == nr[1]
    # two levels: degree 4 then the full degree, the second from the first's series
    d4 = 4
    x2, rep2 = orc.newton_run(s, [d4, s.degree], [2, 2], 0.0, 1e300)
    xl = s.x0[..., :d4 + 1].copy()
    s4 = copy.copy(s)
    s4.degree = d4
    s4.x0 = xl
    for _ in range(2):
        xl, _ = orc.newton_step(s4, xl)
    xf = s.x0.copy()
    xf[..., :d4 + 1] = xl
    for _ in range(2):
        xf, _ = orc.newton_step(s, xf)
    assert np.array_equal(x2, xf) and rep2["iterations"] == [2, 2]


def test_newton_run_rejects_bad_schedules(orc):
    s, x0 = _sqrt_start(2, 8)
    for deg, mi in (([9], [1]), ([4, 2], [1, 1]), ([4], [0]), ([-1], [1])):
        with pytest.raises(RuntimeError):
            orc.newton_run(s, deg, mi, 1e-28, 1.0, x0)


# ------------------------------------------------------------ LU and rcond
def _mat_series(K, rows, d=0, cplx=False):
    """[P][K][d+1][n][n] from exact rows of coefficient 0 (others zero)."""
    n = len(rows)
    P = 2 if cplx else 1
    A = np.zeros((P, K, d + 1, n, n))
    for r in range(n):
        for c in range(n):
            A[0, :, 0, c, r] = mdgen.md_from_fraction(Fraction(rows[r][c]), K)
    return A


def test_lu_needs_and_takes_the_pivot(orc):
    """A_0 = [[0, 1], [1, 1]] has a zero (0,0) entry: only a pivoting LU solves
    it; the solution of A_0 x = (1, 2) is (1, 1) exactly."""
    K = 2
    A = _mat_series(K, [[0, 1], [1, 1]])
    b = np.zeros((1, K, 2, 1))
    b[0, 0, 0, 0], b[0, 0, 1, 0] = 1.0, 2.0
    for method in (0, 1):
        dx = orc.linsolve(K, False, A, b, method=method)
        assert abs(dx[0, 0, 0, 0] - 1.0) <= 1e-30 and abs(dx[0, 0, 1, 0] - 1.0) <= 1e-30, method
    dx = orc.linsolve(K, False, A, b, method=1)
    assert dx[0, 0, 0, 0] == 1.0 and dx[0, 0, 1, 0] == 1.0 and not dx[0, 1].any()


def test_lu_singular_reported(orc):
    A = _mat_series(2, [[1, 2], [2, 4]])
    b = np.ones((1, 2, 2, 1))
    with pytest.raises(RuntimeError):
        orc.linsolve(2, False, A, b, method=1)


@pytest.mark.parametrize("method", [0, 1])
def test_rcond_closed_forms(orc, method):
    """1 / (||A||_1 ||A^-1||_1) for matrices whose inverse is known exactly."""
    K = 4
    # diagonal: min |d_i| / max |d_i|
    assert orc.rcond(K, False, _mat_series(K, [[4, 0, 0], [0, -0.5, 0], [0, 0, 2]]), method) == 0.125
    # unit upper triangular [[1, a], [0, 1]]: inverse [[1, -a], [0, 1]], rcond = 1/(1+|a|)^2
    a = 3.0
    assert orc.rcond(K, False, _mat_series(K, [[1, a], [0, 1]]), method) == pytest.approx(1 / (1 + a) ** 2, rel=1e-15)
    # permutation and scaled identity: 1
    assert orc.rcond(K, False, _mat_series(K, [[0, 0, 1], [1, 0, 0], [0, 1, 0]]), method) == pytest.approx(1.0, rel=1e-15)
    assert orc.rcond(K, False, _mat_series(K, [[7, 0], [0, 7]]), method) == pytest.approx(1.0, rel=1e-15)


def test_rcond_within_norm_equivalence_of_cond2(orc):
    """A_0 = U diag(sigma) V^T with orthogonal U, V and sigma log-spaced on
    [1e-8, 1]: cond_2 = 1e8 up to double rounding of U, V, and the 1-norm
    condition number lies within a factor n of it."""
    n, K = 16, 4
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A0 = U @ np.diag(np.logspace(0, -8, n)) @ V.T
    A = np.zeros((1, K, 1, n, n))
    A[0, 0, 0] = A0.T  # column-major blocks
    for method in (0, 1):
        rc = orc.rcond(K, False, A, method)
        assert 1e-8 / n / 1.001 <= rc <= n * 1e-8 * 1.001, (method, rc)


# ------------------------------------------------------- least squares N > n
@pytest.mark.parametrize("seed,n,N,d,K", [(1, 2, 3, 3, 2), (2, 2, 4, 2, 3), (3, 3, 5, 2, 2)])
def test_lstsq_step_exact_brute_force(orc, seed, n, N, d, K):
    """Whole step of an overdetermined system (N > n, Section 4: least squares)
    against exact rationals: naive AD and each degree's normal equations."""
    s = mdgen.random_system(seed, n=n, K=K, cplx=True, d=d, monos=3, maxvars=2, maxdeg=3, neq=N)
    assert s.N == N
    rng = np.random.default_rng(seed)
    x = s.x0.copy()
    x[:, 0, :, 1:] = rng.uniform(-0.5, 0.5, size=x[:, 0, :, 1:].shape)
    xn, _ = orc.newton_step(s, x)
    xe, dxe, fe, Ae = exact.newton_step_exact(s, x)
    f, A = orc.eval_diff(s, x)
    assert f.shape[2] == N and A.shape[3:] == (n, N)
    for i in range(N):
        for k in range(d + 1):
            a, b = val(f, i, k), fe[i][k]
            sc = 1 + abs(b[0]) + abs(b[1])
            assert abs(a[0] - b[0]) <= 5e4 * eps(K) * sc and abs(a[1] - b[1]) <= 5e4 * eps(K) * sc
    for j in range(n):
        for k in range(d + 1):
            a, b = val(xn, j, k), xe[j][k]
            sc = 1 + abs(b[0]) + abs(b[1])
            assert abs(a[0] - b[0]) <= 1e5 * eps(K) * sc, (j, k, float(a[0] - b[0]))
            assert abs(a[1] - b[1]) <= 1e5 * eps(K) * sc


def test_lstsq_consistent_rows_give_the_square_solution(orc):
    """Appending scaled copies of equations keeps the system consistent: its
    least squares Newton iterates are those of the square system."""
    s = mdgen.config_system(0, 2)
    sa = s.augmented([0, 2, 1], [2.0, -0.5, 4.0])
    assert sa.N == s.n + 3
    x1, n1 = orc.newton(s, 4)
    x2, n2 = orc.newton(sa, 4)
    for j in range(s.n):
        for k in range(s.degree + 1):
            a, b = val(x2, j, k), val(x1, j, k)
            sc = 1 + abs(b[0]) + abs(b[1])
            assert abs(a[0] - b[0]) <= 1e3 * eps(2) * sc and abs(a[1] - b[1]) <= 1e3 * eps(2) * sc


def test_lstsq_linsolve_exact(orc):
    """Block least squares solve (N = 5, n = 3, d = 3) against the exact
    per-degree normal equations."""
    K, N, n, d = 3, 5, 3, 3
    rng = np.random.default_rng(17)
    A = np.zeros((2, K, d + 1, n, N))
    b = np.zeros((2, K, N, d + 1))
    A[:, 0] = rng.standard_normal((2, d + 1, n, N))
    b[:, 0] = rng.standard_normal((2, N, d + 1))
    dx = orc.linsolve(K, True, A, b)
    assert dx.shape == (2, K, n, d + 1)
    dxe = exact.block_lstsq(exact.mat_series_exact(A), exact.vec_series_exact(b))
    for k in range(d + 1):
        for j in range(n):
            a, w = val(dx, j, k), dxe[k][j]
            sc = 1 + abs(w[0]) + abs(w[1])
            assert abs(a[0] - w[0]) <= 1e4 * eps(K) * sc and abs(a[1] - w[1]) <= 1e4 * eps(K) * sc, (k, j)


def test_lstsq_rcond_of_stacked_diagonal(orc):
    """A_0 = [D; 0] (N x n): A_0^+ = [D^-1 0], rcond = min |d_i| / max |d_i|."""
    K = 2
    rows = [[4, 0], [0, -0.5], [0, 0], [0, 0]]
    n, N = 2, 4
    A = np.zeros((1, K, 1, n, N))
    for r in range(N):
        for c in range(n):
            A[0, 0, 0, c, r] = rows[r][c]
    assert orc.rcond(K, False, A) == 0.125
    with pytest.raises(RuntimeError):  # LU needs a square A_0
        orc.rcond(K, False, A, method=1)
