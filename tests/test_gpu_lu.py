"""LU with partial pivoting for A_0 (MD_FLAG_LU) and the 1-norm reciprocal
condition number of A_0 against the oracle.

The LU path feeds the same degree loop as the QR path (W = A_0^-1), so dx
meets the same per-degree tolerance; the Newton step with LU is compared
with the oracle's Newton step with LU; rcond is compared with the oracle's
(both from leading limbs, W computed by different factorisations)."""
import numpy as np
import pytest

import mdgen
from mdcompare import TOL, eps, rel_by_degree, worst_in_eps

pytestmark = pytest.mark.gpu
LU = 0x10


@pytest.fixture(scope="module")
def md():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_06607_gb300 import build

    build.build()
    import paper_2012_06607_gb300 as m

    return m


def _random_linear(K, cplx, n, d, seed, diag=4.0):
    rng = np.random.default_rng(seed)
    P = 2 if cplx else 1
    sc = np.array([2.0 ** (-53 * l) for l in range(K)])
    A = rng.standard_normal((P, K, d + 1, n, n)) * sc[None, :, None, None, None]
    for c in range(n):
        A[0, 0, 0, c, c] += diag
    b = rng.standard_normal((P, K, n, d + 1)) * sc[None, :, None, None]
    return A, b


@pytest.mark.parametrize("K,cplx,n,d", [(2, True, 8, 8), (4, False, 9, 5), (4, True, 33, 6), (8, False, 7, 4),
                                        (1, True, 5, 3), (10, False, 6, 3)])
def test_lu_linsolve_close_to_oracle(md, orc, K, cplx, n, d):
    A, b = _random_linear(K, cplx, n, d, seed=3 * K + n, diag=0.0)  # no diagonal boost: pivoting matters
    ws = md.workspace(md.linsolve_workspace_bytes(K, cplx, n, d, LU))
    Ad, bd = md.to_device(A), md.to_device(b)
    dx = md.linsolve(K, cplx, Ad, bd, ws, flags=LU).cpu().numpy()
    assert md.device_status(ws) == 0
    want = orc.linsolve(K, cplx, A, b, method=1)
    rel = rel_by_degree(dx, want)
    rc = orc.rcond(K, cplx, A, method=1)
    print("lu", K, cplx, n, d, "rcond", rc, "max rel/eps", float((rel / eps(K)).max()))
    for k in range(d + 1):
        assert rel[k] <= TOL * eps(K) * (k + 1), (k, rel[k] / eps(K))
    # rcond of the same A_0 from the device's W
    r = md.linsolve_rcond(K, cplx, Ad, ws, flags=LU)
    assert float(r.item()) == pytest.approx(rc, rel=1e-8)


def test_lu_pivot_needed(md, orc):
    """A_0 = [[0, 1], [1, 1]]: solvable only with a row exchange."""
    K = 2
    A = np.zeros((1, K, 1, 2, 2))
    A[0, 0, 0] = np.array([[0.0, 1.0], [1.0, 1.0]]).T
    b = np.zeros((1, K, 2, 1))
    b[0, 0, :, 0] = [1.0, 2.0]
    ws = md.workspace(md.linsolve_workspace_bytes(K, False, 2, 0, LU))
    dx = md.linsolve(K, False, md.to_device(A), md.to_device(b), ws, flags=LU).cpu().numpy()
    assert md.device_status(ws) == 0
    assert dx[0, 0, 0, 0] == 1.0 and dx[0, 0, 1, 0] == 1.0 and not dx[0, 1].any()


def test_lu_singular_reported(md):
    K = 2
    A = np.zeros((1, K, 1, 2, 2))
    A[0, 0, 0] = np.array([[1.0, 2.0], [2.0, 4.0]]).T
    b = np.ones((1, K, 2, 1))
    ws = md.workspace(md.linsolve_workspace_bytes(K, False, 2, 0, LU))
    md.linsolve(K, False, md.to_device(A), md.to_device(b), ws, flags=LU)
    assert md.device_status(ws) == 4  # MD_ERR_SINGULAR


@pytest.mark.parametrize("flags", [LU, LU | 0x8])
def test_lu_newton_steps(md, orc, flags):
    """cfg0-type system (dd complex n=3, d=8), 4 steps with LU (overlapped and serial)."""
    s = mdgen.config_system(0, 2)
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes(flags))
    x = md.to_device(s.x0)
    xo = s.x0.copy()
    for _ in range(4):
        md.newton_step(sysd, x, ws, flags=flags)
        assert md.device_status(ws) == 0
        xo, _ = orc.newton_step(s, xo, method=1)
    worst = worst_in_eps(x.cpu().numpy(), xo, 2)
    print("lu newton cfg0 flags", flags, "worst rel/eps:", worst)
    assert worst <= TOL


def test_lu_full_size_step(md, orc):
    """Quad double complex n=64, d=64: one step with LU against the oracle's."""
    s = mdgen.config_system(1, 1)
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes(LU))
    x = md.to_device(s.x0)
    md.newton_step(sysd, x, ws, flags=LU)
    assert md.device_status(ws) == 0
    xo, _ = orc.newton_step(s, s.x0, method=1)
    worst = worst_in_eps(x.cpu().numpy(), xo, 4)
    print("lu newton cfg1 worst rel/eps:", worst)
    assert worst <= TOL
    r = md.rcond_a0(sysd, ws, LU)
    A0 = _a0_of(orc, s)
    assert float(r.item()) == pytest.approx(orc.rcond(4, True, A0, method=1), rel=1e-8)


def _a0_of(orc, s):
    _, A = orc.eval_diff(s, s.x0)
    return A


@pytest.mark.parametrize("method", [0, 1])
def test_rcond_after_step_matches_oracle(md, orc, method):
    s = mdgen.config_system(0, 3)
    flags = LU if method else 0
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes(flags))
    x = md.to_device(s.x0)
    md.newton_step(sysd, x, ws, flags=flags)
    r = float(md.rcond_a0(sysd, ws, flags).item())
    want = orc.rcond(s.limbs, True, _a0_of(orc, s), method=method)
    assert r == pytest.approx(want, rel=1e-10)
