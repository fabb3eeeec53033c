"""Seeded synthetic inputs for the power-series Newton step.

This module is shared by the CPU oracle, the tests and the benchmark.  It
holds none of the method's arithmetic: no error-free transformations, no
multiple-double operations, no series products, no solver.  Values are made
exactly with Python integers and ``fractions.Fraction`` and then rounded to
K-limb multiple-double form by greedy nearest-double extraction (each limb is
the correctly rounded residual of the exact value), which yields a
non-overlapping expansion.

Array conventions used throughout the project (P = 2 planes if complex, else
1; K = limbs; n unknowns; d = truncation degree):

* a series vector ``x``:      float64 array ``[P][K][n][d+1]`` (coefficient fastest)
* monomial coefficients:      float64 array ``[P][K][nmono]``
* constant terms:             float64 array ``[P][K][n]``
* matrix series ``A``:        float64 array ``[P][K][d+1][n][n]``, each degree
  block column-major, i.e. index ``[p][l][k][col][row]``.

The system format follows the problem statement of Section 4 (a system
f(x) = 0 of N = n polynomials in x_1..x_n with the series parameter t as the
extra variable, index n).  Each monomial stores up to ``MAXV`` (variable,
exponent) pairs; unused slots hold variable -1 and exponent 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from fractions import Fraction
from typing import List, Optional, Tuple

import numpy as np

MAXV = 4  # (variable, exponent) slots per monomial

# ----------------------------------------------------------------------------
# exact value <-> K-limb expansion


def md_from_fraction(q: Fraction, K: int) -> List[float]:
    """Greedy nearest-double expansion of an exact rational into K limbs."""
    limbs = []
    r = Fraction(q)
    for _ in range(K):
        x = float(r)  # CPython rounds int/int true division correctly
        limbs.append(x)
        r -= Fraction(x)
    return limbs


def md_to_fraction(limbs) -> Fraction:
    """Exact value of an expansion (sum of its limbs)."""
    s = Fraction(0)
    for v in limbs:
        s += Fraction(float(v))
    return s


def fractions_to_md(vals, K: int) -> np.ndarray:
    """List of Fractions -> array [K][len]."""
    out = np.zeros((K, len(vals)))
    for i, q in enumerate(vals):
        out[:, i] = md_from_fraction(q, K)
    return out


def unit_complex(theta: float, K: int) -> Tuple[List[float], List[float]]:
    """cos(theta) + i sin(theta), normalised to unit modulus to ~53K+100 bits.

    The double pair (cos, sin) is divided exactly-enough by its own modulus
    (integer square root), so every limb carries information and the modulus
    of the K-limb result is 1 to about 2^(-53K).
    """
    a, b = math.cos(theta), math.sin(theta)
    A, B = Fraction(a), Fraction(b)
    R2 = A * A + B * B
    N = 53 * K + 100
    num, den = R2.numerator, R2.denominator
    s = math.isqrt(num * den * (1 << (2 * N)))
    r = Fraction(s, den << N)
    return md_from_fraction(A / r, K), md_from_fraction(B / r, K)


def scaled_limbs_value(rng: np.random.Generator, K: int, dist: str = "uniform") -> Fraction:
    """Exact value sum_j u_j 2^(-53 j) with u_j ~ U[-1,1] (or N(0,1))."""
    v = Fraction(0)
    for j in range(K):
        u = rng.uniform(-1.0, 1.0) if dist == "uniform" else rng.standard_normal()
        v += Fraction(float(u)) / (1 << (53 * j))
    return v


# ----------------------------------------------------------------------------
# system container


@dataclass
class System:
    """A polynomial system with md coefficients (host arrays)."""

    limbs: int
    is_complex: bool
    n: int
    degree: int
    poly_ptr: np.ndarray  # int32 [n+1]
    nvar: np.ndarray  # int32 [nmono]
    idx: np.ndarray  # int32 [nmono*MAXV]
    expo: np.ndarray  # int32 [nmono*MAXV]
    coef: np.ndarray  # float64 [P][K][nmono]
    cst: np.ndarray  # float64 [P][K][n]
    x0: np.ndarray  # float64 [P][K][n][d+1], start series (x(0) only)
    seed: Optional[int] = None
    name: str = ""
    meta: dict = field(default_factory=dict)
    neq: int = 0  # number of polynomials N >= n (0: N = n); poly_ptr has N+1 entries, cst N columns

    @property
    def planes(self) -> int:
        return 2 if self.is_complex else 1

    @property
    def N(self) -> int:
        return self.neq if self.neq else self.n

    @property
    def nmono(self) -> int:
        return int(self.nvar.shape[0])

    def monomials(self, i: int):
        """(coef index, [(var, exp), ...]) for polynomial i in CSR order."""
        out = []
        for m in range(self.poly_ptr[i], self.poly_ptr[i + 1]):
            pairs = [(int(self.idx[m * MAXV + q]), int(self.expo[m * MAXV + q])) for q in range(self.nvar[m])]
            out.append((m, pairs))
        return out

    def with_limbs(self, K: int) -> "System":
        """Same exact coefficients re-expanded into K limbs (for 2x-precision references)."""
        P = self.planes

        def conv(arr):
            flat = arr.reshape(P, self.limbs, -1)
            out = np.zeros((P, K, flat.shape[2]))
            for p in range(P):
                for c in range(flat.shape[2]):
                    out[p, :, c] = md_from_fraction(md_to_fraction(flat[p, :, c]), K)
            return out.reshape((P, K) + arr.shape[2:])

        return System(K, self.is_complex, self.n, self.degree, self.poly_ptr.copy(), self.nvar.copy(),
                      self.idx.copy(), self.expo.copy(), conv(self.coef), conv(self.cst), conv(self.x0),
                      self.seed, self.name, dict(self.meta), neq=self.neq)

    def augmented(self, rows, scales) -> "System":
        """Append copies of polynomials rows[r] multiplied by scales[r] (powers of
        two, so the copies are exact): an overdetermined but consistent system
        whose least squares solution is the solution of this one."""
        P, K = self.planes, self.limbs
        pp = [int(v) for v in self.poly_ptr]
        nvar, idx, expo = list(self.nvar), list(self.idx), list(self.expo)
        coef = [self.coef[..., m] for m in range(self.nmono)]
        cst = [self.cst[..., i] for i in range(self.N)]
        for r, sc in zip(rows, scales):
            assert sc != 0 and math.frexp(abs(sc))[0] == 0.5, "scales must be powers of two"
            for m in range(self.poly_ptr[r], self.poly_ptr[r + 1]):
                nvar.append(int(self.nvar[m]))
                idx.extend(int(v) for v in self.idx[m * MAXV:(m + 1) * MAXV])
                expo.extend(int(v) for v in self.expo[m * MAXV:(m + 1) * MAXV])
                coef.append(self.coef[..., m] * sc)
            pp.append(len(nvar))
            cst.append(self.cst[..., r] * sc)
        N = len(pp) - 1
        return System(K, self.is_complex, self.n, self.degree, np.array(pp, np.int32), np.array(nvar, np.int32),
                      np.array(idx, np.int32), np.array(expo, np.int32), np.stack(coef, axis=-1),
                      np.stack(cst, axis=-1), self.x0.copy(), self.seed, self.name + "+ls", dict(self.meta),
                      neq=N)


def _pack(n, K, cplx, d, polys, coefs, csts, x0vals, name="", seed=None, meta=None) -> System:
    """polys: list over i of list of [(var, exp)]; coefs: matching list of (re, im) Fractions.
    len(polys) = N >= n polynomials in n unknowns."""
    P = 2 if cplx else 1
    N = len(polys)
    poly_ptr = [0]
    nvar, idx, expo, cre = [], [], [], []
    for i in range(N):
        for pairs, c in zip(polys[i], coefs[i]):
            assert 0 <= len(pairs) <= MAXV
            nvar.append(len(pairs))
            for q in range(MAXV):
                if q < len(pairs):
                    idx.append(pairs[q][0])
                    expo.append(pairs[q][1])
                else:
                    idx.append(-1)
                    expo.append(0)
            cre.append(c)
        poly_ptr.append(len(nvar))
    nm = len(nvar)
    coef = np.zeros((P, K, nm))
    for m, c in enumerate(cre):
        coef[0, :, m] = md_from_fraction(c[0], K)
        if cplx:
            coef[1, :, m] = md_from_fraction(c[1], K)
    cst = np.zeros((P, K, N))
    for i, c in enumerate(csts):
        cst[0, :, i] = md_from_fraction(c[0], K)
        if cplx:
            cst[1, :, i] = md_from_fraction(c[1], K)
    x0 = np.zeros((P, K, n, d + 1))
    for j, v in enumerate(x0vals):
        x0[0, :, j, 0] = md_from_fraction(v[0], K)
        if cplx:
            x0[1, :, j, 0] = md_from_fraction(v[1], K)
    return System(K, cplx, n, d, np.array(poly_ptr, np.int32), np.array(nvar, np.int32),
                  np.array(idx, np.int32), np.array(expo, np.int32), coef, cst, x0, seed, name, meta or {},
                  neq=N if N != n else 0)


# ----------------------------------------------------------------------------
# exact complex helpers (Fractions) used only to fix constant terms


def _cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def _cpow(a, e):
    r = (Fraction(1), Fraction(0))
    for _ in range(e):
        r = _cmul(r, a)
    return r


def _md_value(limbs_re, limbs_im=None):
    re = md_to_fraction(limbs_re)
    im = md_to_fraction(limbs_im) if limbs_im is not None else Fraction(0)
    return (re, im)


# ----------------------------------------------------------------------------
# random systems (configurations of the benchmark and the tests)


def _random_monomials(rng, n, count, minvars, maxvars, maxdeg, force_t):
    """Distinct monomials over variables 0..n (n = t)."""
    seen = set()
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cannot draw enough distinct monomials")
        m = int(rng.integers(minvars, maxvars + 1))
        m = min(m, maxdeg)
        if force_t and not out:
            others = rng.choice(n, size=m - 1, replace=False) if m > 1 else np.array([], dtype=np.int64)
            vars_ = sorted([int(v) for v in others] + [n])
        else:
            vars_ = sorted(int(v) for v in rng.choice(n + 1, size=m, replace=False))
        D = int(rng.integers(m, maxdeg + 1))
        exps = [1] * m
        for _ in range(D - m):
            exps[int(rng.integers(0, m))] += 1
        key = tuple(zip(vars_, exps))
        if key in seen:
            continue
        seen.add(key)
        out.append(list(key))
    return out


def _jacobian_cond(n, polys, coefs, x0vals):
    """Condition number of the Jacobian at (x0, t=0) in plain double (input sanity check)."""
    x = np.array([complex(float(v[0]), float(v[1])) for v in x0vals])
    J = np.zeros((len(polys), n), dtype=complex)
    for i in range(len(polys)):
        for pairs, c in zip(polys[i], coefs[i]):
            cc = complex(float(c[0]), float(c[1]))
            if any(v == n for v, _ in pairs):
                continue  # vanishes at t = 0 together with its x-derivatives
            for q, (v, e) in enumerate(pairs):
                term = cc * e * x[v] ** (e - 1)
                for q2, (v2, e2) in enumerate(pairs):
                    if q2 != q:
                        term *= x[v2] ** e2
                J[i, v] += term
    return float(np.linalg.cond(J))


def random_system(seed: int, *, n: int, K: int, cplx: bool, d: int, monos: int, minvars: int = 1,
                  maxvars: int, maxdeg: int, coef_kind: str = "unit", cond_max: float = 1e6,
                  name: str = "", neq: int = 0) -> System:
    """Seeded random system whose start point x0 solves it at t = 0.

    neq > n gives N = neq polynomials in n unknowns (all vanish at (x0, 0), so
    the t = 0 system is consistent; for t != 0 it is solved in the least
    squares sense), drawn by the same recipe.

    Recipe: per polynomial, ``monos`` distinct monomials; each draws m ~ U{minvars..maxvars}
    distinct variables among x_1..x_n and t, total degree ~ U{m..maxdeg} with the extra
    units spread uniformly; the first monomial of every polynomial contains t so that the
    solution curve is not constant.  Coefficients are cos(theta) + i sin(theta),
    theta ~ U[0, 2 pi) (complex) or U[-1,1] in the leading limb with lower limbs scaled
    by 2^-53 per limb (real).  The constant term is the exact negated value of the
    remaining monomials at (x0, t = 0), rounded to K limbs.  A draw whose Jacobian at x0
    has condition number above ``cond_max`` is redrawn from the next sub-seed.
    """
    for sub in range(64):
        rng = np.random.default_rng([seed, sub])
        if cplx:
            x0vals = []
            for _ in range(n):
                re, im = unit_complex(float(rng.uniform(0.0, 2 * math.pi)), K)
                x0vals.append((md_to_fraction(re), md_to_fraction(im)))
        else:
            x0vals = []
            for _ in range(n):
                v = scaled_limbs_value(rng, K)
                x0vals.append((md_to_fraction(md_from_fraction(v, K)), Fraction(0)))
        polys, coefs, csts = [], [], []
        xpow_cache = {}
        for i in range(max(n, neq)):
            mons = _random_monomials(rng, n, monos, minvars, maxvars, maxdeg, force_t=True)
            cs = []
            for _ in mons:
                if coef_kind == "unit":
                    re, im = unit_complex(float(rng.uniform(0.0, 2 * math.pi)), K)
                    cs.append((md_to_fraction(re), md_to_fraction(im) if cplx else Fraction(0)))
                else:
                    v = scaled_limbs_value(rng, K)
                    cs.append((md_to_fraction(md_from_fraction(v, K)), Fraction(0)))
            # exact constant: c0 = -sum over monomials without t of c * prod x0^a
            s = (Fraction(0), Fraction(0))
            for pairs, c in zip(mons, cs):
                if any(v == n for v, _ in pairs):
                    continue
                term = c
                for v, e in pairs:
                    key = (v, e)
                    if key not in xpow_cache:
                        xpow_cache[key] = _cpow(x0vals[v], e)
                    term = _cmul(term, xpow_cache[key])
                s = (s[0] + term[0], s[1] + term[1])
            polys.append(mons)
            coefs.append(cs)
            csts.append((-s[0], -s[1]))
        cond = _jacobian_cond(n, polys, coefs, x0vals)
        if cond <= cond_max:
            sysm = _pack(n, K, cplx, d, polys, coefs, csts, x0vals, name=name, seed=seed,
                         meta={"cond_double": cond, "subseed": sub})
            return sysm
    raise RuntimeError("no regular draw found")


# named configurations ---------------------------------------------------------


def config_system(cfg: int, seed: int = 1, **over) -> System:
    """The seeded systems of the workloads.

    0: double double, complex, n=3 (+t), 4 monomials/polynomial of degree <= 2 over 1-2
       variables, d=8.
    1: quad double, complex, n=64 (+t), 64 monomials/polynomial of degree <= 4 over <= 4
       variables, d=64.
    2: octo double, real, n=128 (+t), 32 monomials/polynomial of degree <= 3, d=32.
    """
    if cfg == 0:
        kw = dict(n=3, K=2, cplx=True, d=8, monos=4, minvars=1, maxvars=2, maxdeg=2, coef_kind="unit")
    elif cfg == 1:
        kw = dict(n=64, K=4, cplx=True, d=64, monos=64, minvars=1, maxvars=4, maxdeg=4, coef_kind="unit")
    elif cfg == 2:
        kw = dict(n=128, K=8, cplx=False, d=32, monos=32, minvars=1, maxvars=3, maxdeg=3, coef_kind="uniform")
    else:
        raise ValueError(cfg)
    kw.update(over)
    return random_system(seed, name=f"cfg{cfg}", **kw)


CONFIG_STEPS = {0: 4, 1: 7, 2: 6}


# ----------------------------------------------------------------------------
# systems with closed-form series solutions (pins)


def circle_system(K: int, d: int = 8) -> System:
    """Section 3: t - t^3/6 + t^5/120 - t^7/5040 - y = 0,  x^2 + y^2 - 1 = 0.

    Unknowns x (index 0), y (index 1); t has index 2.  Start point x = 1, y = 0.
    Real coefficients.  The series solution for x is the Taylor series of cos(t)
    through t^8 (y = sin(t) + O(t^9) makes x = cos(t) + O(t^10)).
    """
    n = 2
    F = Fraction
    polys = [
        [[(2, 1)], [(2, 3)], [(2, 5)], [(2, 7)], [(1, 1)]],
        [[(0, 2)], [(1, 2)]],
    ]
    coefs = [
        [(F(1), F(0)), (F(-1, 6), F(0)), (F(1, 120), F(0)), (F(-1, 5040), F(0)), (F(-1), F(0))],
        [(F(1), F(0)), (F(1), F(0))],
    ]
    csts = [(F(0), F(0)), (F(-1), F(0))]
    x0 = [(F(1), F(0)), (F(0), F(0))]
    return _pack(n, K, False, d, polys, coefs, csts, x0, name="circle")


def sqrt_system(K: int, d: int, cplx: bool = False) -> System:
    """x^2 - 1 - t = 0 with x(0) = 1: x(t) = sqrt(1 + t), coefficients binom(1/2, k)."""
    F = Fraction
    polys = [[[(0, 2)], [(1, 1)]]]
    coefs = [[(F(1), F(0)), (F(-1), F(0))]]
    csts = [(F(-1), F(0))]
    x0 = [(F(1), F(0))]
    return _pack(1, K, cplx, d, polys, coefs, csts, x0, name="sqrt1pt")


def binom_half(k: int) -> Fraction:
    """binom(1/2, k) exactly."""
    r = Fraction(1)
    for j in range(k):
        r *= (Fraction(1, 2) - j) / (j + 1)
    return r


def linear_system(seed: int, n: int, K: int, d: int, cplx: bool = True) -> Tuple[System, np.ndarray, np.ndarray, np.ndarray]:
    """(M0 + M1 t) x = c.  Returns (system, M0, M1, c) with exact Fraction entries (object arrays).

    M0 is diagonally dominant so that it is well conditioned.  Monomials: M0[i][j] x_j and
    M1[i][j] x_j t; constant -c_i.  Start point x0 = 0.
    """
    rng = np.random.default_rng([seed, 7])
    F = Fraction

    def rnd():
        re = md_to_fraction(md_from_fraction(scaled_limbs_value(rng, K), K))
        im = md_to_fraction(md_from_fraction(scaled_limbs_value(rng, K), K)) if cplx else F(0)
        return (re, im)

    M0 = [[rnd() for _ in range(n)] for _ in range(n)]
    for i in range(n):
        M0[i][i] = (M0[i][i][0] + 3 * n, M0[i][i][1])
        M0[i][i] = (md_to_fraction(md_from_fraction(M0[i][i][0], K)), M0[i][i][1])
    M1 = [[rnd() for _ in range(n)] for _ in range(n)]
    c = [rnd() for _ in range(n)]
    polys, coefs, csts = [], [], []
    for i in range(n):
        mons, cs = [], []
        for j in range(n):
            mons.append([(j, 1)])
            cs.append(M0[i][j])
        for j in range(n):
            mons.append([(j, 1), (n, 1)])
            cs.append(M1[i][j])
        polys.append(mons)
        coefs.append(cs)
        csts.append((-c[i][0], -c[i][1]))
    x0 = [(F(0), F(0))] * n
    sysm = _pack(n, K, cplx, d, polys, coefs, csts, x0, name="linear")
    return sysm, M0, M1, c


# ----------------------------------------------------------------------------
# random md operands for elementwise tests


def random_md_array(rng: np.random.Generator, K: int, count: int, *, spread: float = 0.0,
                    kind: str = "generic") -> np.ndarray:
    """[K][count] random non-overlapping expansions.

    kind = 'generic': leading limb ~ U[-1,1] * 2^(spread * N(0,1)); lower limbs random.
    """
    out = np.zeros((K, count))
    for c in range(count):
        lead = rng.uniform(-1.0, 1.0) * 2.0 ** (spread * rng.standard_normal())
        v = Fraction(float(lead))
        scale = abs(float(lead))
        for j in range(1, K + 1):
            v += Fraction(float(rng.uniform(-1.0, 1.0) * scale)) / (1 << (53 * j))
        out[:, c] = md_from_fraction(v, K)
    return out


# ----------------------------------------------------------------------------
# linearized solve with an ill-conditioned A_0 (split-product comparison)


def solve_config3(seed: int = 1, n: int = 256, d: int = 16, K: int = 4, cond: float = 1e8):
    """Quad double, real, n = 256, d = 16 block Toeplitz system.

    A_0 = U diag(sigma) V^T with seeded orthogonal U, V (QR of Gaussian matrices,
    in double) and sigma log-spaced on [1/cond, 1]; its double entries are the
    leading limbs.  A_1..A_d and b have N(0,1) leading limbs.  In every matrix
    and vector each lower limb is uniform within half an ulp of the limb above
    it, so every limb is in use; the lower limbs of A_0 move its singular
    values by about 1e-16 times its norm, far below sigma_min = 1/cond.
    Returns (A [1][K][d+1][n][n] column-major blocks, b [1][K][n][d+1]).
    """
    rng = np.random.default_rng([seed, 3])
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sig = np.logspace(0.0, -np.log10(cond), n)
    A0 = (U * sig) @ V.T
    A = np.zeros((1, K, d + 1, n, n))

    def lifted(shape, lead=None):
        # leading limb N(0,1) (or `lead`); limb l uniform in (-ulp/2, ulp/2) of
        # limb l-1, so the expansion is non-overlapping by construction (about
        # 2^-53 per limb)
        out = np.zeros((K,) + shape)
        out[0] = rng.standard_normal(shape) if lead is None else lead
        for l in range(1, K):
            _, e = np.frexp(out[l - 1])
            out[l] = rng.uniform(-0.5, 0.5, size=shape) * np.ldexp(1.0, e - 53)
            out[l][out[l - 1] == 0.0] = 0.0
        return out

    A[0, :, 1:] = lifted((d, n, n))
    A[0, :, 0] = lifted((n, n), lead=A0.T)  # column-major: [col][row]
    b = np.zeros((1, K, n, d + 1))
    b[0] = lifted((n, d + 1))
    return A, b


# ----------------------------------------------------------------------------
# many systems of uneven size for the batched form


def _fixed_unit(rng, size, bits=11):
    """cos t + i sin t, t ~ U[0, 2 pi), each part rounded to `bits` fractional bits."""
    th = rng.uniform(0.0, 2 * math.pi, size)
    sc = float(1 << bits)
    return np.round(np.cos(th) * sc) / sc + 1j * (np.round(np.sin(th) * sc) / sc)


class UnitPool:
    """Full-width unit complex numbers cos t + i sin t, t ~ U[0, 2 pi), made by
    unit_complex (every limb in use, modulus 1 to about 2^(-53K)), with each
    part also held as an exact integer over 2^B, B the finest limb bit of the
    pool.  Draws pick uniformly from the pool: the batched workload takes its
    coefficients from a seeded pool of `size` angles instead of one angle per
    coefficient, which keeps its construction fast."""

    def __init__(self, rng, K: int, size: int):
        self.K = K
        self.limbs = np.zeros((2, K, size))
        for i in range(size):
            re, im = unit_complex(float(rng.uniform(0.0, 2 * math.pi)), K)
            self.limbs[0, :, i] = re
            self.limbs[1, :, i] = im
        # finest bit among all nonzero limbs: value * 2^B is an integer
        nz = self.limbs[self.limbs != 0.0]
        _, ex = np.frexp(nz)
        self.B = int((53 - ex).max())
        self.ints = [self._ints(self.limbs[p]) for p in range(2)]
        self.dbl = self.limbs[0, 0] + 1j * self.limbs[1, 0]

    def _ints(self, limbs):  # [K][size] -> object array of exact integers (value * 2^B)
        out = np.zeros(limbs.shape[1], dtype=object)
        for i in range(limbs.shape[1]):
            v = 0
            for l in range(self.K):
                num, den = float(limbs[l, i]).as_integer_ratio()
                v += num * ((1 << self.B) // den)
            out[i] = v
        return out


def _cmul_obj(ar, ai, br, bi):
    """Exact complex product of object arrays of Python integers."""
    return ar * br - ai * bi, ar * bi + ai * br


def small_system_fast(rng, n: int, d: int, K: int, monos: int, cond_max: float = 1e6, name: str = "",
                      pool: Optional["UnitPool"] = None) -> System:
    """System as in the double-double n=3 configuration but of size n, built fast.

    Per polynomial `monos` distinct monomials of total degree <= 3 over one or two
    variables (t included; the first monomial contains t).

    With a UnitPool (`pool`, K limbs): coefficients and x0 are full-width unit
    complex numbers drawn from the pool, as in the n = 3 configuration, and the
    constant terms are the exact negated values of the t-free monomials at
    (x0, t = 0), computed with Python integers on the pool's power-of-two scale
    and rounded to K limbs, so that x0 solves the system at t = 0.

    Without a pool: coefficients and x0 are cos t + i sin t with real and
    imaginary parts rounded to 11 fractional bits; every product of a
    coefficient with at most three such numbers has at most 44 fractional bits
    and every constant term (a sum of at most `monos` such products, below 2^7
    in modulus) is exact in double, so x0 solves the system at t = 0 exactly.
    Limbs below the leading one are zero.
    """
    N = n + 1
    if pool is not None:
        assert pool.K == K
    for _ in range(64):
        if pool is not None:
            xi = rng.integers(0, pool.dbl.shape[0], n)
            x0 = pool.dbl[xi]
        else:
            x0 = _fixed_unit(rng, n)
        V = np.zeros((n, monos, 2), dtype=np.int64)
        E = np.zeros((n, monos, 2), dtype=np.int64)
        Mv = np.zeros((n, monos), dtype=np.int64)
        todo = np.ones((n, monos), dtype=bool)
        for _round in range(100):
            cnt = int(todo.sum())
            if cnt == 0:
                break
            m = rng.integers(1, 3, cnt)
            v1 = rng.integers(0, N, cnt)
            v2 = rng.integers(0, N - 1, cnt)
            v2 = v2 + (v2 >= v1)
            D = m + rng.integers(0, 4 - m, cnt)  # m..3
            e1 = np.where(m == 1, D, 1 + ((D == 3) & (rng.uniform(size=cnt) < 0.5)))
            e2 = np.where(m == 1, 0, D - e1)
            ii, jj = np.nonzero(todo)
            Mv[ii, jj] = m
            V[ii, jj, 0], V[ii, jj, 1] = v1, v2
            E[ii, jj, 0], E[ii, jj, 1] = e1, e2
            # first monomial of each polynomial contains t
            first = jj == 0
            if first.any():
                rows = ii[first]
                V[rows, 0, 0] = n
                V[rows, 0, 1] = rng.integers(0, n, rows.size)
            # canonical order (smaller variable first) and duplicates
            swap = (Mv == 2) & (V[:, :, 1] < V[:, :, 0])
            V[swap] = V[swap][:, ::-1]
            E[swap] = E[swap][:, ::-1]
            key = np.where(Mv == 1, V[:, :, 0] * 4 + E[:, :, 0],
                           ((V[:, :, 0] * 4 + E[:, :, 0]) * (N + 1) + V[:, :, 1] + 1) * 4 + E[:, :, 1] + 10 ** 9)
            todo[:] = False
            for i in range(n):
                _, first_idx = np.unique(key[i], return_index=True)
                dup = np.ones(monos, dtype=bool)
                dup[first_idx] = False
                todo[i] = dup
        else:
            continue
        if pool is not None:
            ci = rng.integers(0, pool.dbl.shape[0], (n, monos))
            c = pool.dbl[ci]
        else:
            c = _fixed_unit(rng, (n, monos))
        xt = np.concatenate([x0, [0.0]])  # t = 0
        p1 = xt[V[:, :, 0]] ** E[:, :, 0]
        p2 = np.where(Mv == 2, xt[V[:, :, 1]] ** E[:, :, 1], 1.0)
        cst = -(c * p1 * p2).sum(axis=1)
        # Jacobian at (x0, t = 0)
        Jm = np.zeros((n, n), dtype=complex)
        rows = np.repeat(np.arange(n), monos)
        for q in range(2):
            v = V[:, :, q].ravel()
            e = E[:, :, q].ravel()
            ok = (e > 0) & (v < n) & ((q == 0) | (Mv.ravel() == 2))
            other = np.where(q == 0, np.where(Mv == 2, xt[V[:, :, 1]] ** E[:, :, 1], 1.0),
                             xt[V[:, :, 0]] ** E[:, :, 0]).ravel()
            dv = c.ravel() * e * xt[np.minimum(v, n)] ** np.maximum(e - 1, 0) * other
            np.add.at(Jm, (rows[ok], v[ok]), dv[ok])
        if np.linalg.cond(Jm) > cond_max:
            continue
        P = 2
        nm = n * monos
        nvar = Mv.ravel().astype(np.int32)
        idx = np.full((nm, MAXV), -1, dtype=np.int32)
        expo = np.zeros((nm, MAXV), dtype=np.int32)
        idx[:, 0] = V[:, :, 0].ravel()
        expo[:, 0] = E[:, :, 0].ravel()
        two = nvar == 2
        idx[two, 1] = V[:, :, 1].ravel()[two]
        expo[two, 1] = E[:, :, 1].ravel()[two]
        coef = np.zeros((P, K, nm))
        cs = np.zeros((P, K, n))
        xx = np.zeros((P, K, n, d + 1))
        if pool is not None:
            coef[:, :, :] = pool.limbs[:, :, ci.ravel()]
            xx[:, :, :, 0] = pool.limbs[:, :, xi]
            cs[:, :, :] = _exact_constants(pool, xi, ci, V, E, Mv, n)
        else:
            coef[0, 0] = c.real.ravel()
            coef[1, 0] = c.imag.ravel()
            cs[0, 0] = cst.real
            cs[1, 0] = cst.imag
            xx[0, 0, :, 0] = x0.real
            xx[1, 0, :, 0] = x0.imag
        poly_ptr = np.arange(0, nm + 1, monos, dtype=np.int32)
        return System(K, True, n, d, poly_ptr, nvar, idx.ravel(), expo.ravel(), coef, cs, xx, name=name,
                      meta={"cond_double": float(np.linalg.cond(Jm))})
    raise RuntimeError("no regular draw found")


def _exact_constants(pool, xi, ci, V, E, Mv, n):
    """Constant terms [2][K][n]: minus the exact sum, per polynomial, of the
    t-free monomials c x_v1^e1 x_v2^e2 at x0 (t = 0), rounded to K limbs.
    Exact integers: every pool value is an integer over 2^B; a monomial of q
    factors is an integer over 2^(qB), brought to the common scale 2^(4B)."""
    B, K = pool.B, pool.K
    xr = np.append(pool.ints[0][xi], 0).astype(object)  # index n: t = 0
    xim = np.append(pool.ints[1][xi], 0).astype(object)
    one = np.array([1 << B] * (n + 1), dtype=object)
    zero = np.array([0] * (n + 1), dtype=object)
    # powers of every variable at scale 2^(3B): x^0, x^1, x^2, x^3
    pw = [(one * (1 << (2 * B)), zero.copy())]
    cur = (xr, xim)
    for e in (1, 2, 3):
        pw.append((cur[0] << ((3 - e) * B), cur[1] << ((3 - e) * B)))
        if e < 3:
            cur = _cmul_obj(cur[0], cur[1], xr, xim)
    pwr = np.stack([p[0] for p in pw])  # [4][n+1] objects
    pwi = np.stack([p[1] for p in pw])
    v1, e1 = V[:, :, 0], E[:, :, 0]
    v2 = np.where(Mv == 2, V[:, :, 1], n)
    e2 = np.where(Mv == 2, E[:, :, 1], 0)
    # f1 * f2 at scale 2^(6B), times c at 2^B: 2^(7B)
    f1r, f1i = pwr[e1, v1], pwi[e1, v1]
    f2r, f2i = pwr[e2, v2], pwi[e2, v2]
    pr, pi = _cmul_obj(f1r, f1i, f2r, f2i)
    cr, cim = pool.ints[0][ci], pool.ints[1][ci]
    tr, ti = _cmul_obj(pr, pi, cr, cim)
    has_t = (v1 == n) | ((Mv == 2) & (V[:, :, 1] == n))
    tr[has_t] = 0
    ti[has_t] = 0
    sr, si = tr.sum(axis=1), ti.sum(axis=1)
    out = np.zeros((2, K, n))
    den = 1 << (7 * B)
    for i in range(n):
        out[0, :, i] = md_from_fraction(Fraction(-int(sr[i]), den), K)
        out[1, :, i] = md_from_fraction(Fraction(-int(si[i]), den), K)
    return out


def batch_systems(seed: int = 1, count: int = 2048, nmin: int = 8, nmax: int = 64, dmin: int = 8, dmax: int = 32,
                  pool_size: int = 8192):
    """The batched workload: `count` complex systems, n ~ U{nmin..nmax},
    d ~ U{dmin..dmax}, n monomials per polynomial of degree <= 3 over <= 2
    variables, double double or quad double with probability 1/2 each.
    Coefficients and x0 are full-width unit complex numbers (as in the n = 3
    configuration), drawn from a seeded pool of `pool_size` angles per
    precision; constant terms exact (small_system_fast)."""
    rng = np.random.default_rng([seed, 4])
    pools = {K: UnitPool(np.random.default_rng([seed, 5, K]), K, pool_size) for K in (2, 4)}
    out = []
    for b in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        d = int(rng.integers(dmin, dmax + 1))
        K = 2 if rng.uniform() < 0.5 else 4
        out.append(small_system_fast(rng, n, d, K, monos=n, name=f"batch{b}", pool=pools[K]))
    return out
