"""Host-side checks of the C ABI (no GPU needed).

* the library builds for sm_103a, loads, and exports every entry point that
  include/mdnewton.h declares;
* argument validation happens on the host before any CUDA call;
* workspace sizes follow the system structure.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import mdgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(md_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def mdlib():
    from paper_2012_06607_gb300 import build

    build.build()
    import paper_2012_06607_gb300 as md

    return md.lib()


def test_exports_every_declared_symbol(mdlib):
    names = declared_symbols()
    assert len(names) >= 9
    for name in names:
        assert hasattr(mdlib, name), name
    import paper_2012_06607_gb300 as md

    assert set(md.exported_symbols()) <= set(names)


def test_version_and_strings(mdlib):
    assert mdlib.md_version() >= 100
    assert mdlib.md_status_string(4) == b"A_0 is singular"
    assert mdlib.md_status_string(99) == b"unknown status"


def _csys(s, coef_ptr=1, cst_ptr=1):
    import paper_2012_06607_gb300 as md

    pp = np.ascontiguousarray(s.poly_ptr, np.int32)
    nv = np.ascontiguousarray(s.nvar, np.int32)
    ix = np.ascontiguousarray(s.idx, np.int32)
    ex = np.ascontiguousarray(s.expo, np.int32)
    c = md.md_system(s.limbs, int(s.is_complex), s.n, s.degree, s.nmono, pp.ctypes.data, nv.ctypes.data,
                     ix.ctypes.data, ex.ctypes.data, coef_ptr, cst_ptr)
    return c, (pp, nv, ix, ex)


def test_workspace_bytes(mdlib):
    s0 = mdgen.config_system(0, 1)
    c, keep = _csys(s0)
    b0 = mdlib.md_workspace_bytes(ctypes.byref(c), 0)
    assert b0 > 0 and b0 % 256 == 0
    s1 = mdgen.circle_system(2, 8)
    c1, keep1 = _csys(s1)
    b1 = mdlib.md_workspace_bytes(ctypes.byref(c1), 0)
    assert 0 < b1
    # more limbs need more space
    s4 = s0.with_limbs(4)
    c4, keep4 = _csys(s4)
    assert mdlib.md_workspace_bytes(ctypes.byref(c4), 0) > b0
    assert mdlib.md_linsolve_workspace_bytes(4, 1, 64, 64, 0) > mdlib.md_linsolve_workspace_bytes(4, 1, 8, 8, 0) > 0
    assert mdlib.md_linsolve_workspace_bytes(6, 1, 8, 8, 0) == 0  # 6 limbs are not a supported precision


def test_invalid_systems_rejected(mdlib):
    s = mdgen.config_system(0, 1)
    bad_limbs = mdgen.config_system(0, 1)
    bad_limbs.limbs = 7
    c, keep = _csys(bad_limbs)
    assert mdlib.md_workspace_bytes(ctypes.byref(c), 0) == 0
    # variable index out of range
    s2 = mdgen.config_system(0, 1)
    s2.idx = s2.idx.copy()
    s2.idx[0] = s2.n + 1
    c2, keep2 = _csys(s2)
    assert mdlib.md_workspace_bytes(ctypes.byref(c2), 0) == 0
    # repeated variable in one monomial
    s3 = mdgen.config_system(0, 1)
    s3.nvar = s3.nvar.copy()
    s3.idx = s3.idx.copy()
    m = 0
    s3.nvar[m] = 2
    s3.idx[m * 4 + 1] = s3.idx[m * 4]
    s3.expo = s3.expo.copy()
    s3.expo[m * 4 + 1] = 1
    c3, keep3 = _csys(s3)
    assert mdlib.md_workspace_bytes(ctypes.byref(c3), 0) == 0
    # CSR offsets inconsistent with nmono
    s5 = mdgen.config_system(0, 1)
    s5.poly_ptr = s5.poly_ptr.copy()
    s5.poly_ptr[-1] += 1
    c5, keep5 = _csys(s5)
    assert mdlib.md_workspace_bytes(ctypes.byref(c5), 0) == 0
    # a valid one for comparison
    c0, keep0 = _csys(s)
    assert mdlib.md_workspace_bytes(ctypes.byref(c0), 0) > 0


def test_argument_errors_before_cuda(mdlib):
    """Errors detected on the host return without touching the device."""
    assert mdlib.md_elementwise(0, 6, 0, 10, 1, 1, 1, None) == 1  # 6 limbs
    assert mdlib.md_elementwise(9, 2, 0, 10, 1, 1, 1, None) == 1  # unknown op
    assert mdlib.md_elementwise(4, 2, 1, 10, 1, 1, 1, None) == 1  # complex sqrt
    assert mdlib.md_elementwise(0, 2, 0, 10, None, 1, 1, None) == 1
    assert mdlib.md_series_conv(2, 1, -1, 3, 1, 1, 1, None) == 1
    assert mdlib.md_linsolve_series(2, 1, 0, 4, 1, 1, 1, 256, 1 << 20, 0, None) == 1
    assert mdlib.md_linsolve_series(2, 1, 4, 4, 1, 1, 1, None, 1 << 20, 0, None) == 2
    assert mdlib.md_linsolve_series(2, 1, 4, 4, 1, 1, 1, 257, 1 << 20, 0, None) == 2  # misaligned
    assert mdlib.md_linsolve_series(2, 1, 4, 4, 1, 1, 1, 256, 16, 0, None) == 2  # too small
    s = mdgen.config_system(0, 1)
    c, keep = _csys(s)
    assert mdlib.md_newton_series_step(ctypes.byref(c), 1, None, None, 1 << 20, 0, None) == 2
    assert mdlib.md_newton_series_step(ctypes.byref(c), 1, None, 256, 64, 0, None) == 2
    assert mdlib.md_eval_diff(ctypes.byref(c), None, 1, 1, 256, 1 << 30, None) == 1
    assert mdlib.md_get_device_status(None, None) == 2
    mdlib.md_wait_selftest.restype = ctypes.c_int
    mdlib.md_wait_selftest.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]
    assert mdlib.md_wait_selftest(None, 256, 1, None) == 2
    assert mdlib.md_wait_selftest(256, 64, 1, None) == 2  # too small
    assert mdlib.md_wait_selftest(264, 256, 1, None) == 2  # misaligned
    assert mdlib.md_wait_selftest(256, 256, -1, None) == 1


def test_newton_run_host_checks(mdlib):
    """Schedule validation and workspace sizing happen on the host."""
    import paper_2012_06607_gb300 as md

    s = mdgen.config_system(0, seed=1)
    c, keep = _csys(s)
    good = md.schedule([4, s.degree], [3, 3], 1e-28, 1.0)
    wb = mdlib.md_newton_run_workspace_bytes(ctypes.byref(c), ctypes.byref(good), 0)
    assert wb >= mdlib.md_workspace_bytes(ctypes.byref(c), 0) > 0
    for deg, mi, tol in (([s.degree + 1], [1], 0.0), ([4, 2], [1, 1], 0.0), ([4], [0], 0.0),
                         ([4], [1], float("nan")), ([4], [1], -1.0)):
        bad = md.schedule(deg, mi, tol, 1.0)
        assert mdlib.md_newton_run_workspace_bytes(ctypes.byref(c), ctypes.byref(bad), 0) == 0
        st = mdlib.md_newton_series_run(ctypes.byref(c), 256, ctypes.byref(bad), None, 256, 1 << 30, 0, None)
        assert st == 1  # MD_ERR_ARG before any CUDA call
    bad = md.schedule([4], [1])
    bad.nlevels = 0
    assert mdlib.md_newton_run_workspace_bytes(ctypes.byref(c), ctypes.byref(bad), 0) == 0
    # a workspace that is too small or misaligned is refused before any CUDA call
    assert mdlib.md_newton_series_run(ctypes.byref(c), 256, ctypes.byref(good), None, 256, wb - 1, 0, None) == 2
    assert mdlib.md_newton_series_run(ctypes.byref(c), 256, ctypes.byref(good), None, 257, wb, 0, None) == 2
    assert mdlib.md_newton_series_run(ctypes.byref(c), None, ctypes.byref(good), None, 256, wb, 0, None) == 1


def test_lstsq_host_checks(mdlib):
    """N > n: workspace sizes grow with N; shapes and flags are checked on the host."""
    import paper_2012_06607_gb300 as md

    K, n, d = 4, 8, 6
    sq = mdlib.md_lstsq_workspace_bytes(K, 1, n, n, d, 0)
    assert sq == mdlib.md_linsolve_workspace_bytes(K, 1, n, d, 0) > 0
    assert mdlib.md_lstsq_workspace_bytes(K, 1, n + 5, n, d, 0) > sq
    assert mdlib.md_lstsq_workspace_bytes(K, 1, n - 1, n, d, 0) == 0          # N < n
    assert mdlib.md_lstsq_workspace_bytes(K, 1, n + 1, n, d, md.FLAG_LU) == 0  # LU needs N = n
    assert mdlib.md_lstsq_workspace_bytes(K, 1, n + 1, n, d, md.FLAG_OZAKI) == 0
    assert mdlib.md_lstsq_series(K, 1, n - 1, n, d, 256, 256, 256, 256, 1 << 30, 0, None) == 1
    assert mdlib.md_lstsq_series(K, 1, n + 1, n, d, 256, 256, 256, 256, 1 << 30, md.FLAG_LU, None) == 1
    assert mdlib.md_lstsq_series(K, 1, n + 1, n, d, 256, 256, 256, 256, 1 << 30, md.FLAG_OZAKI, None) == 8
    # systems: neq rows
    s = mdgen.config_system(0, seed=1)
    sa = s.augmented([0, 1], [2.0, 0.5])
    c, keep = _csys(s)
    ca, keepa = _csys(sa)
    ca.neq = sa.N
    assert mdlib.md_workspace_bytes(ctypes.byref(ca), 0) > mdlib.md_workspace_bytes(ctypes.byref(c), 0)
    assert mdlib.md_workspace_bytes(ctypes.byref(ca), md.FLAG_LU) == 0
    ca.neq = s.n - 1  # fewer equations than unknowns
    assert mdlib.md_workspace_bytes(ctypes.byref(ca), 0) == 0
    ca.neq = sa.N
    arr = (md.md_system * 1)(ca)
    assert mdlib.md_batched_workspace_bytes(1, arr, 0) == 0  # the batched form is square only


def test_python_flags_match_header():
    import re

    import paper_2012_06607_gb300 as md

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mdnewton.h")).read()
    defs = {k: int(v, 0) for k, v in re.findall(r"#define\s+(MD_\w+)\s+(0x[0-9a-fA-F]+|\d+)\b", hdr)}
    for name in ("OZAKI", "AUTOTUNE", "GRAPH", "SERIAL", "LU", "PHASE_TIMES", "CHECK"):
        assert getattr(md, "FLAG_" + name) == defs["MD_FLAG_" + name], name
    assert md.PHASE_STAMPS == defs["MD_PHASE_STAMPS"] == len(md.PHASE_NAMES) + 1


def test_batched_job_costs_host_only():
    """md_batched_job_costs needs no device: K^2 and complex x4 scaling, growth
    with the degree, and argument errors."""
    import paper_2012_06607_gb300 as md

    base = mdgen.config_system(0, 1)  # double double complex, n = 3, d = 8
    c2 = md.batched_job_costs([base])[0]
    c4 = md.batched_job_costs([base.with_limbs(4)])[0]
    assert c2 > 0 and c4 == pytest.approx(4.0 * c2)
    rng = np.random.default_rng(3)
    lo = mdgen.small_system_fast(rng, 6, 4, 2, monos=6)
    hi = mdgen.small_system_fast(np.random.default_rng(3), 6, 12, 2, monos=6)
    cl, ch = md.batched_job_costs([lo, hi])
    assert ch > cl
    arr = (md.md_system * 1)()
    assert md.lib().md_batched_job_costs(0, arr, None) == 1  # MD_ERR_ARG


def test_plan_cache_collision_replans_host_only():
    """Structures whose hashes collide (the test hook narrows every hash to one
    value) each get their own plan: the host cost estimate of every system,
    computed from its plan, equals its value with the full hash, whether the
    colliding systems come in one call or in turns."""
    import paper_2012_06607_gb300 as md

    systems = [mdgen.config_system(0, 1), mdgen.config_system(0, 2),
               mdgen.small_system_fast(np.random.default_rng(4), 6, 5, 2, monos=6),
               mdgen.small_system_fast(np.random.default_rng(5), 9, 7, 4, monos=9)]
    want = md.batched_job_costs(systems)
    assert len(set(want)) == len(want)  # distinct structures, distinct costs
    L = md.lib()
    try:
        L.md_plan_cache_hash_mask(1)  # every structure hashes to the same key
        assert np.array_equal(md.batched_job_costs(systems), want)
        for _ in range(2):
            for s, w in zip(systems, want):
                assert md.batched_job_costs([s])[0] == w
    finally:
        L.md_plan_cache_hash_mask(0)
    assert np.array_equal(md.batched_job_costs(systems), want)


def test_batched_plan_cache_bound_host_only():
    """Workspace queries over many distinct batches (new coefficient pointers
    each time) stay correct while the batch plan cache drops old entries."""
    import paper_2012_06607_gb300 as md

    systems = [mdgen.config_system(0, 1), mdgen.small_system_fast(np.random.default_rng(2), 5, 4, 2, monos=5)]
    keep = []
    sizes = []
    for _ in range(40):
        arr = (md.md_system * len(systems))()
        for i, s in enumerate(systems):
            arr[i] = md._host_md_system(s, keep)  # fresh host copies: new pointers, new key
        sizes.append(md.lib().md_batched_workspace_bytes(len(systems), arr, 0))
    assert sizes[0] > 0 and len(set(sizes)) == 1


def test_plan_check_fuzz_host_only():
    """Bounds mode on the host: the plans of many seeded systems (shapes,
    degrees, limbs, real and complex, N > n, the split-product layout) pass
    every table and layout check; an invalid system is an argument error."""
    import paper_2012_06607_gb300 as md

    rng = np.random.default_rng(11)
    count = 0
    for seed in range(40):
        n = int(rng.integers(1, 12))
        K = int(rng.choice([1, 2, 3, 4, 5, 8, 10]))
        d = int(rng.integers(0, 12))
        maxvars = min(int(rng.integers(1, 5)), n + 1)
        try:
            s = mdgen.random_system(seed, n=n, K=K, cplx=bool(seed % 2), d=d, monos=int(rng.integers(1, 4)),
                                    maxvars=maxvars, maxdeg=maxvars + int(rng.integers(0, 3)), coef_kind="uniform",
                                    cond_max=1e30, neq=n + int(rng.integers(0, 3)) if seed % 3 == 0 else 0)
        except RuntimeError:  # no regular Jacobian for this shape: nothing to plan
            continue
        flags = md.FLAG_OZAKI if (seed % 4 == 1 and s.N == s.n) else 0
        assert md.plan_check(s, flags) == 0, (seed, n, K, d)
        count += 1
    for cfg in range(5):
        s = mdgen.config_system(cfg, 1) if cfg != 3 and cfg != 4 else None
        if s is not None:
            assert md.plan_check(s) == 0, cfg
    assert count >= 20  # 23 of the 40 seeded shapes are regular
    bad = mdgen.config_system(0, 1)
    keep = []
    c = md._host_md_system(bad, keep)
    c.n = 0  # invalid
    assert md.lib().md_plan_check(ctypes.byref(c), 0) == 1  # MD_ERR_ARG
    assert md.lib().md_status_string(9) == b"bounds check failed"


def test_split_form_workspace_host_only():
    """MD_FLAG_OZAKI lays out fixed-point copies (the series pool; for the
    batched form also A and dx) only from three limbs on: the split-form
    workspace grows at K = 4 by at least the pool copy, and the batched
    double-double workspace is the same in both forms."""
    import paper_2012_06607_gb300 as md

    keep = []
    s2 = mdgen.small_system_fast(np.random.default_rng(3), 6, 5, 2, monos=6)
    s4 = s2.with_limbs(4)
    lib = md.lib()
    for s, grows in ((s2, False), (s4, True)):
        arr = (md.md_system * 1)()
        arr[0] = md._host_md_system(s, keep)
        plain = lib.md_batched_workspace_bytes(1, arr, 0)
        split = lib.md_batched_workspace_bytes(1, arr, md.FLAG_OZAKI)
        assert plain > 0 and split > 0
        if grows:
            n, d = s.n, s.degree
            words = ((53 * 4 + 31) // 32 + 2 + 4) & ~3  # packed 32-bit words per plane value
            copy_A = 4 * 2 * words * (d + 1) * n * n
            assert split >= plain + copy_A
        else:
            assert split == plain
    c4 = md._host_md_system(s4, keep)
    assert lib.md_workspace_bytes(ctypes.byref(c4), md.FLAG_OZAKI) > lib.md_workspace_bytes(ctypes.byref(c4), 0)


def test_plan_factor_sms_without_plan_host_only():
    """md_plan_factor_sms reports -1 for a structure and form no step has
    planned, and for an invalid structure (host-only lookups)."""
    import paper_2012_06607_gb300 as md

    keep = []
    s = mdgen.small_system_fast(np.random.default_rng(11), 7, 5, 4, monos=7)
    c = md._host_md_system(s, keep)
    lib = md.lib()
    assert lib.md_plan_factor_sms(ctypes.byref(c), 0) == -1
    assert lib.md_plan_factor_sms(ctypes.byref(c), md.FLAG_OZAKI) == -1
    bad = md._host_md_system(s, keep)
    bad.limbs = 6  # not a supported precision
    assert lib.md_plan_factor_sms(ctypes.byref(bad), 0) == -1
