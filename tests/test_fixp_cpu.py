"""The fixed-point scalar arithmetic of the Householder chain (csrc/fixp.cuh),
compiled for the host, against exact rationals: conversion from K limbs and
back, products, sums (with cancellation), reciprocal square roots, square
roots and reciprocals, each within a few units of 2^(-53K) relative to the
exact result.  The conversion to K limbs must give non-overlapping limbs."""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import mdgen

HERE = os.path.dirname(os.path.abspath(__file__))
KS = [2, 3, 4, 5, 8, 10]


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("fixp") / "fixp_host.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", os.path.join(HERE, "fixp_host.cpp"),
                           "-o", so])
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    lib.fxp_op.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, P, P, P]
    return lib


def _call(fx, K, op, x, y=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    yp = None if y is None else np.ascontiguousarray(y, dtype=np.float64).ctypes.data
    assert fx.fxp_op(K, op, x.shape[0], x.ctypes.data, yp, out.ctypes.data) == 0
    return out


def _val(limbs):
    return sum((Fraction(float(v)) for v in limbs), Fraction(0))


def _operands(K, count, seed, positive=False):
    rng = np.random.default_rng([K, seed])
    x = mdgen.random_md_array(rng, K, count, spread=40.0).T.copy()  # [count][K]
    if positive:
        x *= np.sign(x[:, :1])
    return x


def _nonoverlapping(limbs):
    for a, b in zip(limbs[:-1], limbs[1:]):
        if b != 0.0:
            assert a != 0.0 and abs(b) < abs(a) * 2.0 ** -52 * 2, (a, b)


def _rel(got, want):
    return abs(got - want) / abs(want)


@pytest.mark.parametrize("K", KS)
def test_round_trip_and_products(fx, K):
    x, y = _operands(K, 300, 1), _operands(K, 300, 2)
    tol = Fraction(8) * Fraction(2) ** (-53 * K)
    rt = _call(fx, K, 0, x)
    pr = _call(fx, K, 1, x, y)
    for i in range(x.shape[0]):
        X, Y = _val(x[i]), _val(y[i])
        assert _rel(_val(rt[i]), X) <= tol, (K, i)
        assert _rel(_val(pr[i]), X * Y) <= tol, (K, i)
        _nonoverlapping(rt[i])
        _nonoverlapping(pr[i])


@pytest.mark.parametrize("K", KS)
def test_sums_with_cancellation(fx, K):
    x = _operands(K, 300, 3)
    y = _operands(K, 300, 4)
    # a third of the pairs cancel in their leading limbs (y = -x_0 + x_tail / 2,
    # a valid expansion), a third cancel exactly
    y[:100, 0] = -x[:100, 0]
    y[:100, 1:] = x[:100, 1:] * 0.5
    y[100:200] = -x[100:200]
    s = _call(fx, K, 2, x, y)
    for i in range(x.shape[0]):
        want = _val(x[i]) + _val(y[i])
        got = _val(s[i])
        # truncation below the last word of the larger operand
        bound = Fraction(8) * Fraction(2) ** (-53 * K) * max(abs(_val(x[i])), abs(_val(y[i])))
        assert abs(got - want) <= bound, (K, i)


@pytest.mark.parametrize("K", KS)
def test_square_roots_and_reciprocals(fx, K):
    a = _operands(K, 200, 5, positive=True)
    tol = Fraction(16) * Fraction(2) ** (-53 * K)
    rs = _call(fx, K, 3, a)
    sq = _call(fx, K, 4, a)
    rc = _call(fx, K, 5, a)
    for i in range(a.shape[0]):
        A = _val(a[i])
        assert _rel(_val(rs[i]) ** 2 * A, Fraction(1)) <= 2 * tol, (K, i, "rsqrt")
        assert _rel(_val(sq[i]) ** 2, A) <= 2 * tol, (K, i, "sqrt")
        assert _rel(_val(rc[i]) * A, Fraction(1)) <= tol, (K, i, "recip")
        _nonoverlapping(sq[i])


@pytest.mark.parametrize("K", [2, 4, 8])
def test_non_finite_values_propagate(fx, K):
    """A non-finite limb anywhere gives NaN limbs after any operation, and the
    reciprocal (square root) of zero is not finite, as in md arithmetic."""
    x = _operands(K, 4, 7, positive=True)
    y = x.copy()
    y[0, 0] = np.inf
    y[1, K - 1] = np.nan
    y[2, 0] = -np.inf
    for op in (0, 1, 2):
        out = _call(fx, K, op, x, y) if op else _call(fx, K, op, y)
        for i in range(3):
            assert np.isnan(out[i]).all(), (K, op, i)
        if op:
            assert np.isfinite(out[3]).all()
    z = np.zeros((2, K))
    for op in (3, 5):
        assert not np.isfinite(_call(fx, K, op, z)).any(), (K, op)


@pytest.mark.parametrize("K", [2, 4])
def test_products_round_to_nearest(fx, K):
    """The conversion back to K limbs rounds the last limb to nearest: the
    signed error of many products, in units of the last limb's place, averages
    near zero (a truncation would average about -1/2) and never reaches 1."""
    x, y = _operands(K, 1500, 11, positive=True), _operands(K, 1500, 12, positive=True)
    pr = _call(fx, K, 1, x, y)
    errs = []
    for i in range(x.shape[0]):
        want = _val(x[i]) * _val(y[i])
        last = pr[i, K - 1]
        if last == 0.0:
            continue
        ulp = Fraction(2) ** (int(np.frexp(abs(last))[1]) - 53)
        errs.append(float((_val(pr[i]) - want) / ulp))
    errs = np.array(errs)
    assert len(errs) > 1000
    assert np.abs(errs).max() <= 0.5 + 1e-3, np.abs(errs).max()
    assert abs(errs.mean()) < 0.05, errs.mean()
