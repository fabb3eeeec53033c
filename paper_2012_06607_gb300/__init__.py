"""GB300 library for the power-series Newton step in multiple-double arithmetic.

Thin Python binding over the C ABI of ``libmdnewton.so`` (``include/mdnewton.h``).
Every step of the computation runs in the library's CUDA kernels; this module
only marshals arguments: PyTorch provides device memory and streams.  There is
no CPU fallback -- importing the binding without the built library, or calling
it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdnewton.so")

MAXV = 4
STATUS = {0: "MD_OK", 1: "MD_ERR_ARG", 2: "MD_ERR_WORKSPACE", 3: "MD_ERR_CUDA", 4: "MD_ERR_SINGULAR",
          5: "MD_ERR_NONFINITE", 6: "MD_ERR_NOCONV", 7: "MD_ERR_TIMEOUT", 8: "MD_ERR_UNSUPPORTED"}
OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4, "mul_d": 5}


class MdError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)}")


class md_system(ctypes.Structure):
    _fields_ = [("limbs", ctypes.c_int), ("is_complex", ctypes.c_int), ("n", ctypes.c_int), ("degree", ctypes.c_int),
                ("nmono", ctypes.c_int), ("poly_ptr", ctypes.c_void_p), ("nvar", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("expo", ctypes.c_void_p), ("coef", ctypes.c_void_p),
                ("cst", ctypes.c_void_p), ("neq", ctypes.c_int)]


MAX_LEVELS = 16


class md_newton_schedule(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int), ("degree", ctypes.c_int * MAX_LEVELS),
                ("max_iter", ctypes.c_int * MAX_LEVELS), ("tol", ctypes.c_double), ("too_large", ctypes.c_double)]


class md_newton_report(ctypes.Structure):
    _fields_ = [("levels_done", ctypes.c_int), ("converged", ctypes.c_int),
                ("iterations", ctypes.c_int * MAX_LEVELS), ("dx_norm", ctypes.c_double * MAX_LEVELS),
                ("dx_max", ctypes.c_double * MAX_LEVELS)]


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2012_06607_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, sz, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_longlong
        L.md_version.restype = i
        L.md_status_string.restype = ctypes.c_char_p
        L.md_status_string.argtypes = [i]
        L.md_workspace_bytes.restype = sz
        L.md_workspace_bytes.argtypes = [ctypes.POINTER(md_system), i]
        L.md_linsolve_workspace_bytes.restype = sz
        L.md_linsolve_workspace_bytes.argtypes = [i, i, i, i, i]
        L.md_elementwise.argtypes = [i, i, i, ll, vp, vp, vp, vp]
        L.md_series_conv.argtypes = [i, i, i, ll, vp, vp, vp, vp]
        L.md_eval_diff.argtypes = [ctypes.POINTER(md_system), vp, vp, vp, vp, sz, vp]
        L.md_linsolve_series.argtypes = [i, i, i, i, vp, vp, vp, vp, sz, i, vp]
        L.md_newton_series_step.argtypes = [ctypes.POINTER(md_system), vp, vp, vp, sz, i, vp]
        L.md_get_device_status.argtypes = [vp, vp]
        L.md_batched_workspace_bytes.argtypes = [i, ctypes.POINTER(md_system), i]
        L.md_batched_workspace_bytes.restype = sz
        L.md_batched_job_costs.argtypes = [i, ctypes.POINTER(md_system), ctypes.c_void_p]
        L.md_batched_job_costs.restype = i
        L.md_plan_check.argtypes = [ctypes.POINTER(md_system), i]
        L.md_plan_check.restype = i
        L.md_newton_series_step_batched.argtypes = [i, ctypes.POINTER(md_system), ctypes.POINTER(vp), vp, vp, vp, sz,
                                                    i, vp]
        L.md_newton_series_step_batched.restype = i
        L.md_linsolve_series_static.argtypes = [i, i, i, i, vp, vp, vp, i, vp]
        L.md_linsolve_series_static.restype = i
        L.md_profile_enable.argtypes = [i]
        L.md_profile_enable.restype = None
        L.md_profile_read.argtypes = [vp, vp, i]
        L.md_profile_read.restype = i
        L.md_profile_kind_name.argtypes = [i]
        L.md_profile_kind_name.restype = ctypes.c_char_p
        sched_p, rep_p = ctypes.POINTER(md_newton_schedule), ctypes.POINTER(md_newton_report)
        L.md_newton_run_workspace_bytes.argtypes = [ctypes.POINTER(md_system), sched_p, i]
        L.md_newton_run_workspace_bytes.restype = sz
        L.md_newton_series_run.argtypes = [ctypes.POINTER(md_system), vp, sched_p, rep_p, vp, sz, i, vp]
        L.md_rcond_a0.argtypes = [ctypes.POINTER(md_system), vp, sz, i, vp, vp]
        L.md_linsolve_rcond.argtypes = [i, i, i, i, vp, vp, sz, i, vp, vp]
        L.md_lstsq_workspace_bytes.argtypes = [i, i, i, i, i, i]
        L.md_lstsq_workspace_bytes.restype = sz
        L.md_lstsq_series.argtypes = [i, i, i, i, i, vp, vp, vp, vp, sz, i, vp]
        L.md_lstsq_rcond.argtypes = [i, i, i, i, i, vp, vp, sz, i, vp, vp]
        L.md_wait_selftest.argtypes = [vp, sz, i, vp]
        L.md_plan_cache_hash_mask.argtypes = [ctypes.c_ulonglong]
        L.md_plan_cache_hash_mask.restype = None
        L.md_plan_factor_sms.argtypes = [ctypes.POINTER(md_system), i]
        L.md_plan_factor_sms.restype = i
        for name in ("md_elementwise", "md_series_conv", "md_eval_diff", "md_linsolve_series",
                     "md_newton_series_step", "md_get_device_status", "md_newton_series_run", "md_rcond_a0",
                     "md_linsolve_rcond", "md_lstsq_series", "md_lstsq_rcond", "md_wait_selftest"):
            getattr(L, name).restype = i
        _lib = L
    return _lib


def exported_symbols():
    return ["md_version", "md_status_string", "md_workspace_bytes", "md_linsolve_workspace_bytes",
            "md_elementwise", "md_series_conv", "md_eval_diff", "md_linsolve_series",
            "md_newton_series_step", "md_get_device_status", "md_batched_workspace_bytes",
            "md_newton_series_step_batched", "md_linsolve_series_static", "md_profile_enable",
            "md_profile_read", "md_profile_kind_name", "md_newton_run_workspace_bytes", "md_newton_series_run",
            "md_rcond_a0", "md_linsolve_rcond", "md_lstsq_workspace_bytes", "md_lstsq_series", "md_lstsq_rcond",
            "md_batched_job_costs", "md_plan_check", "md_wait_selftest", "md_plan_cache_hash_mask",
            "md_plan_factor_sms"]


# --------------------------------------------------------------- helpers
def _torch():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("paper_2012_06607_gb300 needs a CUDA device")
    return torch


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check(code: int, what: str):
    if code != 0:
        raise MdError(code, what)


def to_device(a: np.ndarray, device="cuda"):
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)


def workspace(nbytes: int, device="cuda"):
    torch = _torch()
    return torch.zeros(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ------------------------------------------------------------- the system
class DeviceSystem:
    """A system with host structure arrays and device coefficient arrays.

    ``s`` is any object with the fields of ``md_system`` as numpy arrays
    (poly_ptr, nvar, idx, expo int32; coef [P][K][nmono], cst [P][K][N] float64)
    and optionally ``neq`` (N polynomials, 0 or absent: N = n).
    """

    def __init__(self, s, device="cuda"):
        self.limbs, self.is_complex, self.n, self.degree = int(s.limbs), bool(s.is_complex), int(s.n), int(s.degree)
        self.poly_ptr = np.ascontiguousarray(s.poly_ptr, dtype=np.int32)
        self.nvar = np.ascontiguousarray(s.nvar, dtype=np.int32)
        self.idx = np.ascontiguousarray(s.idx, dtype=np.int32)
        self.expo = np.ascontiguousarray(s.expo, dtype=np.int32)
        self.nmono = int(self.nvar.shape[0])
        self.coef = to_device(s.coef, device)
        self.cst = to_device(s.cst, device)
        self.neq = int(getattr(s, "neq", 0) or 0)
        self._c = md_system(self.limbs, int(self.is_complex), self.n, self.degree, self.nmono,
                            self.poly_ptr.ctypes.data, self.nvar.ctypes.data if self.nmono else None,
                            self.idx.ctypes.data if self.nmono else None, self.expo.ctypes.data if self.nmono else None,
                            _ptr(self.coef) if self.nmono else None, _ptr(self.cst), self.neq)

    @property
    def planes(self):
        return 2 if self.is_complex else 1

    def c(self):
        return ctypes.byref(self._c)

    def workspace_bytes(self, flags: int = 0) -> int:
        return int(lib().md_workspace_bytes(self.c(), flags))


# ------------------------------------------------------------ entry points
def elementwise(op: str, limbs: int, is_complex: bool, x, y=None, out=None, stream=None):
    """x, y: CUDA tensors [P][K][count] (y: [count] doubles for mul_d)."""
    z = out if out is not None else x.new_empty(x.shape)
    count = x.shape[-1]
    _check(lib().md_elementwise(OPS[op], limbs, int(is_complex), count, _ptr(x), _ptr(y), _ptr(z), _stream(stream)),
           "md_elementwise")
    return z


def series_conv(limbs: int, is_complex: bool, x, y, out=None, stream=None):
    """x, y: CUDA tensors [P][K][count][d+1]."""
    z = out if out is not None else x.new_empty(x.shape)
    _check(lib().md_series_conv(limbs, int(is_complex), x.shape[-1] - 1, x.shape[2], _ptr(x), _ptr(y), _ptr(z),
                                _stream(stream)), "md_series_conv")
    return z


def eval_diff(sysd: DeviceSystem, x, ws, f=None, A=None, stream=None):
    torch = _torch()
    P, K, n, d = sysd.planes, sysd.limbs, sysd.n, sysd.degree
    N = sysd.neq or n
    f = f if f is not None else torch.empty((P, K, N, d + 1), dtype=torch.float64, device=x.device)
    A = A if A is not None else torch.empty((P, K, d + 1, n, N), dtype=torch.float64, device=x.device)
    _check(lib().md_eval_diff(sysd.c(), _ptr(x), _ptr(f), _ptr(A), _ptr(ws), ws.numel(), _stream(stream)),
           "md_eval_diff")
    return f, A


def linsolve_workspace_bytes(limbs: int, is_complex: bool, n: int, degree: int, flags: int = 0) -> int:
    return int(lib().md_linsolve_workspace_bytes(limbs, int(is_complex), n, degree, flags))


def linsolve(limbs: int, is_complex: bool, A, b, ws, dx=None, flags: int = 0, stream=None):
    """A: [P][K][d+1][n][n], b: [P][K][n][d+1] CUDA tensors -> dx like b."""
    n, d = b.shape[2], b.shape[3] - 1
    dx = dx if dx is not None else b.new_empty(b.shape)
    _check(lib().md_linsolve_series(limbs, int(is_complex), n, d, _ptr(A), _ptr(b), _ptr(dx), _ptr(ws), ws.numel(),
                                    flags, _stream(stream)), "md_linsolve_series")
    return dx


def newton_step(sysd: DeviceSystem, x, ws, dx_norm=None, flags: int = 0, stream=None):
    """In-place step on x ([P][K][n][d+1] CUDA tensor); dx_norm: CUDA double[2] or None.
    flags: FLAG_OZAKI (the split-product form; size ws with the same flag),
    FLAG_LU, FLAG_SERIAL, FLAG_CHECK, FLAG_AUTOTUNE (the factorisation's SM
    count tuned over the plan's first calls; see plan_factor_sms)."""
    _check(lib().md_newton_series_step(sysd.c(), _ptr(x), _ptr(dx_norm), _ptr(ws), ws.numel(), flags,
                                       _stream(stream)), "md_newton_series_step")
    return x


FLAG_OZAKI, FLAG_AUTOTUNE, FLAG_GRAPH, FLAG_SERIAL, FLAG_LU = 0x1, 0x2, 0x4, 0x8, 0x10
FLAG_PHASE_TIMES = 0x20  # batched form: times is [nsys, PHASE_STAMPS]
FLAG_CHECK = 0x40  # bounds mode: plan tables and workspace layout checked on the host (MD_ERR_CHECK)
PHASE_STAMPS = 10
PHASE_NAMES = ("load", "products", "accumulation", "qr_setup", "householder_qr", "rinv", "w", "degree_loop",
               "finish")


def rcond_a0(sysd: DeviceSystem, ws, flags: int = 0, out=None, stream=None):
    """1-norm reciprocal condition number of A_0 of the last newton_step on ws
    (CUDA double tensor [1], written asynchronously)."""
    torch = _torch()
    out = out if out is not None else torch.empty(1, dtype=torch.float64, device=ws.device)
    _check(lib().md_rcond_a0(sysd.c(), _ptr(ws), ws.numel(), flags, _ptr(out), _stream(stream)), "md_rcond_a0")
    return out


def lstsq_workspace_bytes(limbs: int, is_complex: bool, neq: int, n: int, degree: int, flags: int = 0) -> int:
    return int(lib().md_lstsq_workspace_bytes(limbs, int(is_complex), neq, n, degree, flags))


def lstsq(limbs: int, is_complex: bool, A, b, ws, dx=None, flags: int = 0, stream=None):
    """Least squares block Toeplitz solve: A [P][K][d+1][n][N], b [P][K][N][d+1]
    CUDA tensors -> dx [P][K][n][d+1]."""
    n, N, d = A.shape[3], A.shape[4], A.shape[2] - 1
    dx = dx if dx is not None else b.new_empty((b.shape[0], b.shape[1], n, d + 1))
    _check(lib().md_lstsq_series(limbs, int(is_complex), N, n, d, _ptr(A), _ptr(b), _ptr(dx), _ptr(ws), ws.numel(),
                                 flags, _stream(stream)), "md_lstsq_series")
    return dx


def lstsq_rcond(limbs: int, is_complex: bool, A, ws, flags: int = 0, out=None, stream=None):
    """1 / (||A_0||_1 ||A_0^+||_1) after lstsq(A) on ws."""
    torch = _torch()
    n, N, d = A.shape[3], A.shape[4], A.shape[2] - 1
    out = out if out is not None else torch.empty(1, dtype=torch.float64, device=ws.device)
    _check(lib().md_lstsq_rcond(limbs, int(is_complex), N, n, d, _ptr(A), _ptr(ws), ws.numel(), flags, _ptr(out),
                                _stream(stream)), "md_lstsq_rcond")
    return out


def linsolve_rcond(limbs: int, is_complex: bool, A, ws, flags: int = 0, out=None, stream=None):
    """Same for the A_0 of the last linsolve(A) on ws."""
    torch = _torch()
    n, d = A.shape[3], A.shape[2] - 1
    out = out if out is not None else torch.empty(1, dtype=torch.float64, device=ws.device)
    _check(lib().md_linsolve_rcond(limbs, int(is_complex), n, d, _ptr(A), _ptr(ws), ws.numel(), flags, _ptr(out),
                                   _stream(stream)), "md_linsolve_rcond")
    return out


def schedule(degrees, max_iter, tol: float = 1e-32, too_large: float = 1.0) -> md_newton_schedule:
    """Degree-continuation schedule for newton_run (levels of equal length lists)."""
    if len(degrees) != len(max_iter) or not 1 <= len(degrees) <= MAX_LEVELS:
        raise ValueError("degrees and max_iter: 1..16 levels of equal length")
    sc = md_newton_schedule()
    sc.nlevels = len(degrees)
    for l, (d, m) in enumerate(zip(degrees, max_iter)):
        sc.degree[l] = int(d)
        sc.max_iter[l] = int(m)
    sc.tol = float(tol)
    sc.too_large = float(too_large)
    return sc


def newton_run_workspace_bytes(sysd: DeviceSystem, sched: md_newton_schedule, flags: int = 0) -> int:
    return int(lib().md_newton_run_workspace_bytes(sysd.c(), ctypes.byref(sched), flags))


def newton_run(sysd: DeviceSystem, x, ws, sched: md_newton_schedule, flags: int = 0, stream=None) -> dict:
    """Newton with degree continuation on x ([P][K][n][D+1] CUDA tensor, in
    place).  Returns {levels_done, converged, iterations, dx_norm, dx_max}."""
    rep = md_newton_report()
    _check(lib().md_newton_series_run(sysd.c(), _ptr(x), ctypes.byref(sched), ctypes.byref(rep), _ptr(ws),
                                      ws.numel(), flags, _stream(stream)), "md_newton_series_run")
    L = rep.levels_done
    return {"levels_done": L, "converged": bool(rep.converged), "iterations": list(rep.iterations[:L]),
            "dx_norm": list(rep.dx_norm[:L]), "dx_max": list(rep.dx_max[:L])}


def _sys_array(systems):
    arr = (md_system * len(systems))()
    for i, sd in enumerate(systems):
        arr[i] = sd._c
    return arr


def _host_md_system(s, keep) -> "md_system":
    """md_system over host arrays of any object with its fields (the host
    planning reads the structure only; coef and cst are never read there)."""
    pp = np.ascontiguousarray(s.poly_ptr, dtype=np.int32)
    nv = np.ascontiguousarray(s.nvar, dtype=np.int32)
    ix = np.ascontiguousarray(s.idx, dtype=np.int32)
    ex = np.ascontiguousarray(s.expo, dtype=np.int32)
    cf = np.ascontiguousarray(s.coef, dtype=np.float64)
    cs = np.ascontiguousarray(s.cst, dtype=np.float64)
    keep += [pp, nv, ix, ex, cf, cs]
    nm = int(nv.shape[0])
    return md_system(int(s.limbs), int(bool(s.is_complex)), int(s.n), int(s.degree), nm, pp.ctypes.data,
                     nv.ctypes.data if nm else None, ix.ctypes.data if nm else None, ex.ctypes.data if nm else None,
                     cf.ctypes.data if nm else None, cs.ctypes.data, int(getattr(s, "neq", 0) or 0))


def plan_check(system, flags: int = 0) -> int:
    """md_plan_check: the bounds mode's host checks on one system's plan
    (DeviceSystem, or any object with the md_system fields); returns the status."""
    keep = []
    c = system._c if hasattr(system, "_c") else _host_md_system(system, keep)
    return int(lib().md_plan_check(ctypes.byref(c), flags))


def batched_job_costs(systems) -> np.ndarray:
    """md_batched_job_costs: the host cost estimate of each system's step
    (DeviceSystem, or any object with the md_system fields as arrays)."""
    keep = []
    arr = (md_system * len(systems))()
    for i, sd in enumerate(systems):
        arr[i] = sd._c if hasattr(sd, "_c") else _host_md_system(sd, keep)
    out = np.zeros(len(systems), dtype=np.float64)
    _check(lib().md_batched_job_costs(len(systems), arr, out.ctypes.data), "md_batched_job_costs")
    return out


def shard_lpt(costs, world: int):
    """Partition of a batch over `world` GPUs, longest processing time first:
    systems in decreasing cost (ties: lower index), each to the rank with the
    least total cost so far (ties: lower rank).  Returns per rank its system
    indices in that order.  Deterministic, so every rank computes the same
    partition without communicating."""
    import heapq

    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return out


def batched_workspace_bytes(systems, flags: int = 0) -> int:
    return int(lib().md_batched_workspace_bytes(len(systems), _sys_array(systems), flags))


def newton_step_batched(systems, xs, ws, dx_norm=None, times=None, flags: int = 0, stream=None):
    """One Newton step for every system (DeviceSystem list) on its series xs[i]
    (CUDA tensors, updated in place).  dx_norm: CUDA double [nsys, 2] or None;
    times: CUDA int64 [nsys, 2] (global-timer ns at start/end) or None;
    [nsys, PHASE_STAMPS] with FLAG_PHASE_TIMES (start, the end of each phase
    of PHASE_NAMES)."""
    arr = _sys_array(systems)
    xp = (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])
    _check(lib().md_newton_series_step_batched(len(systems), arr, xp, _ptr(dx_norm), _ptr(times), _ptr(ws),
                                               ws.numel(), flags, _stream(stream)), "md_newton_series_step_batched")
    return xs


def device_status(ws, stream=None) -> int:
    return int(lib().md_get_device_status(_ptr(ws), _stream(stream)))


def plan_factor_sms(sysd: DeviceSystem, flags: int = 0) -> int:
    """md_plan_factor_sms: the tuned SM count of the factorisation in the
    cached plan of this system and form (0 while untuned, -1 if no plan)."""
    return int(lib().md_plan_factor_sms(sysd.c(), int(flags)))


def wait_selftest(ws, target: int, stream=None) -> None:
    """Runs the library's bounded device wait on a counter nothing increments
    (md_wait_selftest); read the outcome with device_status."""
    _check(lib().md_wait_selftest(_ptr(ws), ws.numel(), int(target), _stream(stream)), "md_wait_selftest")


# ------------------------------------------------------------------ profiling
def profile_enable(on: bool = True) -> None:
    lib().md_profile_enable(int(on))


def profile_read() -> dict:
    """{kernel class: (milliseconds, launches)} since the last read (synchronises)."""
    n = 32
    ms = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    k = lib().md_profile_read(ms.ctypes.data, cnt.ctypes.data, n)
    if k < 0:
        raise RuntimeError("md_profile_read failed")
    return {lib().md_profile_kind_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(k) if cnt[i]}
