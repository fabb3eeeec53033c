"""The allocation-free solve (md_linsolve_series_static) against md_linsolve_series.

md_linsolve_series_static serves callers that cannot allocate a device
workspace (device memory owned by another allocator or reserved to the limit,
code where cudaMalloc/cudaFree would synchronise the device, contexts that
forbid allocation): it runs the same solve in a static 16 MiB device array of
the library.  It runs the same kernels on the same workspace layout, so two
calls in a row with different systems must each give exactly the bits of the
workspace entry point (and so lie within the solve tests' tolerance), with the
QR, LU and split-product forms; a singular A_0 shows as non-finite entries of
dx; oversize requests are refused before any device work.  Collected last on
purpose, and self-contained so that it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from mdcompare import md_diff, md_value, modulus

pytestmark = pytest.mark.gpu


def eps(K):
    return 2.0 ** (-52 * K)


@pytest.fixture(scope="module")
def md():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_06607_gb300 import build

    build.build()
    import paper_2012_06607_gb300 as m

    return m


def _system(K, cplx, n, d, seed):
    rng = np.random.default_rng(seed)
    P = 2 if cplx else 1
    sc = np.array([2.0 ** (-53 * l) for l in range(K)])
    A = rng.standard_normal((P, K, d + 1, n, n)) * sc[None, :, None, None, None]
    for c in range(n):
        A[0, 0, 0, c, c] += 4.0
    b = rng.standard_normal((P, K, n, d + 1)) * sc[None, :, None, None]
    return A, b


def _static_solve(md, K, cplx, A, b, flags=0):
    import torch

    Ad, bd = md.to_device(A), md.to_device(b)
    dx = torch.empty_like(bd)
    n, d = b.shape[2], b.shape[3] - 1
    st = md.lib().md_linsolve_series_static(K, int(cplx), n, d, Ad.data_ptr(), bd.data_ptr(), dx.data_ptr(), flags,
                                             torch.cuda.current_stream().cuda_stream)
    assert st == 0, st
    torch.cuda.synchronize()
    return dx.cpu().numpy()


def _reference_solve(md, K, cplx, A, b, flags=0):
    n, d = b.shape[2], b.shape[3] - 1
    ws = md.workspace(md.linsolve_workspace_bytes(K, cplx, n, d, flags))
    dx = md.linsolve(K, cplx, md.to_device(A), md.to_device(b), ws, flags=flags).cpu().numpy()
    assert md.device_status(ws) == 0
    return dx


def _check_close(got, want, K):
    diff = modulus(md_diff(got, want))
    scale = np.maximum(modulus(md_value(want)).max(axis=0), 1e-300)
    rel = diff.max(axis=0) / scale
    for k in range(rel.shape[0]):
        assert rel[k] <= 1e3 * eps(K) * (k + 1), (k, rel[k] / eps(K))


LU, OZAKI = 0x10, 0x1


@pytest.mark.parametrize("flags", [0, LU, OZAKI])
def test_static_matches_workspace_entry_point_twice(md, flags):
    cases = [(4, True, 16, 12, 1), (2, False, 24, 9, 2)]
    for K, cplx, n, d, seed in cases:  # two calls in a row, different systems
        A, b = _system(K, cplx, n, d, seed)
        got = _static_solve(md, K, cplx, A, b, flags)
        want = _reference_solve(md, K, cplx, A, b, flags)
        assert np.array_equal(got, want), (flags, K, n, d)
        _check_close(got, want, K)


@pytest.mark.parametrize("flags", [0, LU])
@pytest.mark.parametrize("col", [0, 3, 7])
def test_static_singular_gives_nonfinite_dx(md, flags, col):
    """A_0 with one exactly zero column (first, middle, last): the status word
    is not readable on this path, so the header promises non-finite entries
    in dx instead.  The workspace entry point reports MD_ERR_SINGULAR for the
    same A_0."""
    K, cplx, n, d = 2, True, 8, 3
    A, b = _system(K, cplx, n, d, 11 + col)
    A[:, :, 0, col, :] = 0.0
    got = _static_solve(md, K, cplx, A, b, flags)
    assert not np.isfinite(got).all(), (flags, col)
    ws = md.workspace(md.linsolve_workspace_bytes(K, cplx, n, d, flags))
    md.linsolve(K, cplx, md.to_device(A), md.to_device(b), ws, flags=flags)
    assert md.device_status(ws) == 4  # MD_ERR_SINGULAR
    # and the next call on the shared array is clean again
    A2, b2 = _system(K, cplx, n, d, 5)
    assert np.array_equal(_static_solve(md, K, cplx, A2, b2, flags), _reference_solve(md, K, cplx, A2, b2, flags))


def test_static_rejects_oversize(md):
    L = md.lib()
    n, d = 512, 64  # needs far more than the 16 MiB scratch
    assert L.md_linsolve_workspace_bytes(4, 1, n, d, 0) > (16 << 20)
    st = L.md_linsolve_series_static(4, 1, n, d, ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256), 0,
                                      None)
    assert st == 2  # MD_ERR_WORKSPACE, nothing launched
    assert L.md_linsolve_series_static(6, 1, 8, 8, ctypes.c_void_p(256), ctypes.c_void_p(256), ctypes.c_void_p(256),
                                       0, None) == 1
