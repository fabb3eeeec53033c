"""Split-product (Ozaki) form against the oracle.

The form computes r_k = b_k - sum_j A_{k-j} dx_j from exact slice products on
the BF16 tensor pipe with exact fixed-point accumulation and one rounding to
K limbs, and (in the Newton step) the series products of the evaluation on
32-bit word slices with exact products and column sums.  It must meet the same
per-degree tolerance as the plain form, and on the ill-conditioned
quad-double system (n = 256, d = 16, cond(A_0) = 1e8) its error against the
oracle must not exceed the plain form's (equal accuracy).
"""
import numpy as np
import pytest

import mdgen
from mdcompare import TOL, eps, rel_by_degree, worst_in_eps

pytestmark = pytest.mark.gpu

OZAKI = 1


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


def _solve(md, K, cplx, A, b, flags):
    n, d = b.shape[2], b.shape[3] - 1
    ws = md.workspace(md.linsolve_workspace_bytes(K, cplx, n, d, flags))
    dx = md.linsolve(K, cplx, md.to_device(A), md.to_device(b), ws, flags=flags).cpu().numpy()
    assert md.device_status(ws) == 0
    return dx


@pytest.mark.parametrize("K,cplx,n,d", [(2, True, 8, 8), (4, False, 9, 5), (4, True, 16, 12), (8, False, 7, 4),
                                        (3, True, 33, 3), (5, False, 20, 6), (10, True, 6, 3), (1, False, 5, 6)])
def test_ozaki_linsolve_close_to_oracle(md, orc, K, cplx, n, d):
    A, b = _random_linear(K, cplx, n, d, seed=K * 7 + n)
    got = _solve(md, K, cplx, A, b, OZAKI)
    want = orc.linsolve(K, cplx, A, b)
    rel = rel_by_degree(got, want)
    print("ozaki linsolve", K, cplx, n, d, "max rel/eps:", float((rel / eps(K)).max()))
    for k in range(d + 1):
        assert rel[k] <= 1e3 * eps(K) * (k + 1), (k, rel[k] / eps(K))


def test_ozaki_newton_steps(md, orc):
    import torch

    for s, steps in ((mdgen.config_system(0, 1), 4), (mdgen.sqrt_system(4, 16), 5)):
        sysd = md.DeviceSystem(s)
        ws = md.workspace(sysd.workspace_bytes(OZAKI))
        x = md.to_device(s.x0)
        xo = s.x0.copy()
        for _ in range(steps):
            md.newton_step(sysd, x, ws, flags=OZAKI)
            assert md.device_status(ws) == 0
            xo, _ = orc.newton_step(s, xo)
        worst = worst_in_eps(x.cpu().numpy(), xo, s.limbs)
        print(s.name, "ozaki newton worst rel/eps:", worst)
        assert worst <= TOL


@pytest.mark.parametrize("K,cplx", [(3, True), (5, False), (8, True), (10, False), (2, False)])
def test_ozaki_newton_other_precisions(md, orc, K, cplx):
    """The split-product form (series products on 32-bit word slices, update
    on 8-bit slices) at other limb counts: four steps of a random system
    against the oracle's, per degree within 1e3 eps_K."""
    import torch

    s = mdgen.random_system(60 + K, n=6, K=K, cplx=cplx, d=10, monos=5, maxvars=3, maxdeg=3,
                            coef_kind="unit" if cplx else "uniform", name=f"oz{K}")
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes(OZAKI))
    x = md.to_device(s.x0)
    xo = s.x0.copy()
    for _ in range(4):
        md.newton_step(sysd, x, ws, flags=OZAKI)
        assert md.device_status(ws) == 0
        xo, _ = orc.newton_step(s, xo)
    worst = worst_in_eps(x.cpu().numpy(), xo, K)
    print("ozaki K", K, cplx, "worst rel/eps:", worst)
    assert worst <= TOL


def test_ozaki_octo_double_full_size_step(md, orc):
    """Octo double real, n = 128, d = 32: one split-product step against the
    oracle's and against the deca double oracle on the same exact inputs."""
    s = mdgen.config_system(2, 1)
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes(OZAKI))
    x = md.to_device(s.x0)
    md.newton_step(sysd, x, ws, flags=OZAKI)
    assert md.device_status(ws) == 0
    xo, _ = orc.newton_step(s, s.x0)
    worst = worst_in_eps(x.cpu().numpy(), xo, 8)
    ref = s.with_limbs(10)
    xr, _ = orc.newton_step(ref, ref.x0)
    worst2 = worst_in_eps(x.cpu().numpy(), xr, 8)
    print("cfg2 ozaki step worst rel/eps: oracle", worst, "deca double", worst2)
    assert worst <= TOL and worst2 <= TOL


def test_ozaki_full_size_newton_step(md, orc):
    """Quad double complex n = 64, d = 64: one step with the split-product update."""
    s = mdgen.config_system(1, 1)
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes(OZAKI))
    x = md.to_device(s.x0)
    md.newton_step(sysd, x, ws, flags=OZAKI)
    assert md.device_status(ws) == 0
    xo, _ = orc.newton_step(s, s.x0)
    worst = worst_in_eps(x.cpu().numpy(), xo, 4)
    print("cfg1 ozaki step worst rel/eps:", worst)
    assert worst <= TOL
    # and against the oracle with twice the limbs on the same exact inputs
    xr, _ = orc.newton_step(s.with_limbs(8), s.with_limbs(8).x0)
    worst2 = worst_in_eps(x.cpu().numpy(), xr, 4)
    print("cfg1 ozaki step against octo double: worst rel/eps:", worst2)
    assert worst2 <= TOL


def test_ill_conditioned_solve_equal_accuracy(md, orc):
    """Quad double real n = 256, d = 16, cond(A_0) = 1e8: split-product and plain
    forms against the oracle, degree by degree."""
    A, b = mdgen.solve_config3(1)
    K = 4
    want = orc.linsolve(K, False, A, b)
    plain = _solve(md, K, False, A, b, 0)
    oz = _solve(md, K, False, A, b, OZAKI)
    rp = rel_by_degree(plain, want)
    ro = rel_by_degree(oz, want)
    print("cfg3 rel err vs oracle per degree (plain):", [f"{v:.1e}" for v in rp])
    print("cfg3 rel err vs oracle per degree (ozaki):", [f"{v:.1e}" for v in ro])
    for k in range(b.shape[3]):
        assert ro[k] <= 10.0 * rp[k] + 1e3 * eps(K), (k, ro[k], rp[k])
