"""CPU oracle for the multiple-double power-series Newton step.

TEST INFRASTRUCTURE ONLY.  Imported by ``tests/``, by ``__graft_entry__.smoke``
and by the benchmark's ``cpu_baseline`` / ``--impl reference`` arm; the product
package never imports it.  The C sources (``mdoracle.c``) share no code with
the CUDA library.  ``build()`` compiles two shared objects from the same file:
the plain oracle and an op-counting variant (``-DORACLE_COUNT``) that counts
every binary64 operation for the Table 1 and Section 3 cost pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mdoracle.c")
LIB = os.path.join(HERE, "libmdoracle.so")
LIB_COUNT = os.path.join(HERE, "libmdoracle_count.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC", "-std=c11"]

_lock = threading.Lock()
_libs = {}


def build(force: bool = False) -> None:
    """Compile the oracle (plain and counting variants) with gcc."""
    # the counting variant is serial: its global counters are not thread-safe
    for out, flags in ((LIB, CFLAGS), (LIB_COUNT, [f for f in CFLAGS if f != "-fopenmp"] + ["-DORACLE_COUNT"])):
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
            tmp = out + ".tmp%d" % os.getpid()
            subprocess.check_call(["gcc", *flags, SRC, "-o", tmp, "-lm"])
            os.replace(tmp, out)


def _load(counting: bool):
    key = bool(counting)
    with _lock:
        if key not in _libs:
            build()
            lib = ctypes.CDLL(LIB_COUNT if counting else LIB)
            P = ctypes.c_void_p
            i = ctypes.c_int
            lib.orc_md_op.argtypes = [i, i, i, ctypes.c_long, P, P, P]
            lib.orc_series_conv.argtypes = [i, i, i, ctypes.c_long, P, P, P]
            lib.orc_eval_diff.argtypes = [i, i, i, i, i, P, P, P, P, P, P, P, P, P]
            lib.orc_linsolve.argtypes = [i, i, i, i, P, P, P, P]
            lib.orc_linsolve_m.argtypes = [i, i, i, i, P, P, P, P, i]
            lib.orc_lstsq.argtypes = [i, i, i, i, i, P, P, P, P, i]
            lib.orc_eval_diff_ls.argtypes = [i, i, i, i, i, i, P, P, P, P, P, P, P, P, P]
            lib.orc_newton_step_m.argtypes = [i, i, i, i, i, P, P, P, P, P, P, P, P, P, i]
            lib.orc_newton_step_ls.argtypes = [i, i, i, i, i, i, P, P, P, P, P, P, P, P, P, i]
            lib.orc_rcond.argtypes = [i, i, i, i, i, P, i, P]
            lib.orc_newton_step.argtypes = [i, i, i, i, i, P, P, P, P, P, P, P, P, P]
            d = ctypes.c_double
            lib.orc_newton_run.argtypes = [i, i, i, i, i, i, P, P, P, P, P, P, P, i, P, P, d, d, P, P, P, i]
            lib.orc_count_get.argtypes = [P]
            lib.orc_set_threads.argtypes = [i]
            _libs[key] = lib
        return _libs[key]


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st == 4:
        raise OracleError(f"{what}: singular A_0")
    if st != 0:
        raise OracleError(f"{what}: status {st}")


OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4, "mul_d": 5}


class Oracle:
    """ctypes front end.  Arrays follow the layouts documented in ``mdgen``."""

    def __init__(self, counting: bool = False, threads: int = 0):
        self.lib = _load(counting)
        if threads:
            self.lib.orc_set_threads(threads)

    def threads(self) -> int:
        return int(self.lib.orc_set_threads(0))

    # -- op counts ------------------------------------------------------
    def count_reset(self):
        self.lib.orc_count_reset()

    def counts(self) -> dict:
        out = np.zeros(10, dtype=np.int64)
        self.lib.orc_count_get(_p(out))
        keys = ["add", "sub", "mul", "div", "fma", "sqrt", "twoprod", "series_mul", "series_add", "twosum"]
        return dict(zip(keys, [int(v) for v in out]))

    # -- elementwise ----------------------------------------------------
    def md_op(self, op: str, K: int, cplx: bool, x: np.ndarray, y: Optional[np.ndarray] = None) -> np.ndarray:
        """x, y: [P][K][count] (y: [count] doubles for mul_d)."""
        x = _f64(x)
        count = x.shape[-1]
        z = np.zeros_like(x)
        yy = _f64(y) if y is not None else None
        _check(self.lib.orc_md_op(OPS[op], K, int(cplx), count, _p(x), _p(yy), _p(z)), "md_op")
        return z

    def series_conv(self, K: int, cplx: bool, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        """x, y: [P][K][count][d+1]."""
        x, y = _f64(x), _f64(y)
        z = np.zeros_like(x)
        d = x.shape[-1] - 1
        _check(self.lib.orc_series_conv(K, int(cplx), d, x.shape[2], _p(x), _p(y), _p(z)), "series_conv")
        return z

    # -- the method -----------------------------------------------------
    def _sysargs(self, s):
        return (_i32(s.poly_ptr), _i32(s.nvar), _i32(s.idx), _i32(s.expo), _f64(s.coef), _f64(s.cst))

    def eval_diff(self, s, x: np.ndarray):
        """Returns (f [P][K][N][d+1], A [P][K][d+1][n][N] column-major blocks);
        N = number of polynomials (N >= n)."""
        P, K, n, d, N = s.planes, s.limbs, s.n, s.degree, s.N
        pp, nv, ix, ex, cf, cs = self._sysargs(s)
        x = _f64(x)
        f = np.zeros((P, K, N, d + 1))
        A = np.zeros((P, K, d + 1, n, N))
        st = self.lib.orc_eval_diff_ls(K, int(s.is_complex), N, n, d, s.nmono, _p(pp), _p(nv), _p(ix), _p(ex), _p(cf),
                                       _p(cs), _p(x), _p(f), _p(A))
        _check(st, "eval_diff")
        return f, A

    def linsolve(self, K: int, cplx: bool, A: np.ndarray, b: np.ndarray, want_rdiag: bool = False, method: int = 0):
        """A: [P][K][d+1][n][N] (col-major blocks), b: [P][K][N][d+1] -> dx
        [P][K][n][d+1]; least squares when N > n.  method 0: Householder QR
        of A_0, 1: LU with partial pivoting (N = n)."""
        A, b = _f64(A), _f64(b)
        P, _, D1, n, N = A.shape
        dx = np.zeros((P, K, n, D1))
        rd = np.zeros(n)
        _check(self.lib.orc_lstsq(K, int(cplx), N, n, D1 - 1, _p(A), _p(b), _p(dx), _p(rd), method), "linsolve")
        return (dx, rd) if want_rdiag else dx

    def rcond(self, K: int, cplx: bool, A: np.ndarray, method: int = 0) -> float:
        """1 / (||A_0||_1 ||A_0^-1||_1) from the leading limbs; A as for linsolve."""
        A = _f64(A)
        P, _, D1, n, N = A.shape
        out = np.zeros(1)
        _check(self.lib.orc_rcond(K, int(cplx), N, n, D1 - 1, _p(A), method, _p(out)), "rcond")
        return float(out[0])

    def newton_step(self, s, x: np.ndarray, want_rdiag: bool = False, method: int = 0):
        """One step; returns (x_new, (|dx_d|, |dx|_inf))."""
        P, K, n, d = s.planes, s.limbs, s.n, s.degree
        pp, nv, ix, ex, cf, cs = self._sysargs(s)
        xx = _f64(x).copy()
        nrm = np.zeros(2)
        rd = np.zeros(n)
        st = self.lib.orc_newton_step_ls(K, int(s.is_complex), s.N, n, d, s.nmono, _p(pp), _p(nv), _p(ix), _p(ex),
                                         _p(cf), _p(cs), _p(xx), _p(nrm), _p(rd), method)
        _check(st, "newton_step")
        if want_rdiag:
            return xx, (float(nrm[0]), float(nrm[1])), rd
        return xx, (float(nrm[0]), float(nrm[1]))

    def newton_run(self, s, degrees, max_iter, tol: float, too_large: float, x: Optional[np.ndarray] = None,
                   method: int = 0):
        """Newton with degree continuation (Sec. 6).  Returns (x, report) with
        report = {levels_done, iterations, dx_norm, dx_max, converged}."""
        P, K, n, D = s.planes, s.limbs, s.n, s.degree
        pp, nv, ix, ex, cf, cs = self._sysargs(s)
        xx = _f64(s.x0 if x is None else x).copy()
        nlev = len(degrees)
        dg = np.asarray(degrees, dtype=np.int32)
        mi = np.asarray(max_iter, dtype=np.int32)
        it = np.zeros(nlev, dtype=np.int32)
        dxn = np.zeros(2 * nlev)
        lv = np.zeros(1, dtype=np.int32)
        st = self.lib.orc_newton_run(K, int(s.is_complex), s.N, n, D, s.nmono, _p(pp), _p(nv), _p(ix), _p(ex), _p(cf),
                                     _p(cs), _p(xx), nlev, _p(dg), _p(mi), ctypes.c_double(tol),
                                     ctypes.c_double(too_large), _p(it), _p(dxn), _p(lv), method)
        _check(st, "newton_run")
        L = int(lv[0])
        rep = {"levels_done": L, "iterations": [int(v) for v in it[:L]],
               "dx_norm": [float(v) for v in dxn[0:2 * L:2]], "dx_max": [float(v) for v in dxn[1:2 * L:2]]}
        rep["converged"] = all(v <= tol for v in rep["dx_norm"])
        return xx, rep

    def newton(self, s, steps: int, x: Optional[np.ndarray] = None):
        x = s.x0.copy() if x is None else x
        norms = []
        for _ in range(steps):
            x, nr = self.newton_step(s, x)
            norms.append(nr)
        return x, norms
