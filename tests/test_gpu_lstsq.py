"""Least squares (N > n equations, Section 4) on the GPU against the oracle:
the block solve with a tall A_0, Newton steps of overdetermined systems
(consistent ones give the square system's iterates), the pseudo-inverse
condition number, and the host-side refusals (LU, split products)."""
import numpy as np
import pytest

import mdgen
from mdcompare import TOL, eps, rel_by_degree, worst_in_eps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_06607_gb300 import build

    build.build()
    import paper_2012_06607_gb300 as m

    return m


def _tall(K, cplx, N, n, d, seed):
    rng = np.random.default_rng(seed)
    P = 2 if cplx else 1
    sc = np.array([2.0 ** (-53 * l) for l in range(K)])
    A = rng.standard_normal((P, K, d + 1, n, N)) * sc[None, :, None, None, None]
    b = rng.standard_normal((P, K, N, d + 1)) * sc[None, :, None, None]
    return A, b


@pytest.mark.parametrize("K,cplx,N,n,d", [(2, True, 12, 8, 6), (4, False, 40, 33, 4), (4, True, 70, 64, 3),
                                          (8, False, 9, 5, 3), (1, True, 7, 3, 5), (3, True, 135, 128, 1)])
def test_lstsq_close_to_oracle(md, orc, K, cplx, N, n, d):
    A, b = _tall(K, cplx, N, n, d, seed=N + 7 * n + K)
    ws = md.workspace(md.lstsq_workspace_bytes(K, cplx, N, n, d))
    Ad, bd = md.to_device(A), md.to_device(b)
    dx = md.lstsq(K, cplx, Ad, bd, ws).cpu().numpy()
    assert md.device_status(ws) == 0
    assert dx.shape == (2 if cplx else 1, K, n, d + 1)
    want = orc.linsolve(K, cplx, A, b)
    rc = orc.rcond(K, cplx, A)
    rel = rel_by_degree(dx, want)
    print("lstsq", K, cplx, N, n, d, "rcond", rc, "max rel/eps", float((rel / eps(K)).max()))
    for k in range(d + 1):
        assert rel[k] <= TOL * eps(K) * (k + 1), (k, rel[k] / eps(K))
    r = md.lstsq_rcond(K, cplx, Ad, ws)
    assert float(r.item()) == pytest.approx(rc, rel=1e-8)


def test_consistent_overdetermined_newton(md, orc):
    """Scaled copies of equations appended: the GPU's least squares steps match
    the oracle's and the square system's."""
    s = mdgen.config_system(0, 2)
    sa = s.augmented([0, 2, 1], [2.0, -0.5, 4.0])
    xs = {}
    for sys_ in (s, sa):
        sysd = md.DeviceSystem(sys_)
        ws = md.workspace(sysd.workspace_bytes())
        x = md.to_device(sys_.x0)
        for _ in range(4):
            md.newton_step(sysd, x, ws)
            assert md.device_status(ws) == 0
        xs[sys_.N] = x.cpu().numpy()
    xo, _ = orc.newton(sa, 4)
    w1, w2 = worst_in_eps(xs[sa.N], xo, 2), worst_in_eps(xs[sa.N], xs[s.n], 2)
    print("consistent ls newton worst rel/eps: vs oracle", w1, "vs square system", w2)
    assert w1 <= TOL and w2 <= TOL


@pytest.mark.parametrize("seed,n,N,cplx,K,d", [(1, 3, 5, True, 2, 8), (2, 6, 9, False, 4, 6), (3, 16, 20, True, 4, 12)])
def test_overdetermined_newton_steps(md, orc, seed, n, N, cplx, K, d):
    s = mdgen.random_system(seed, n=n, K=K, cplx=cplx, d=d, monos=4, minvars=1, maxvars=3, maxdeg=3, neq=N)
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    x = md.to_device(s.x0)
    xo = s.x0.copy()
    for _ in range(3):
        md.newton_step(sysd, x, ws)
        assert md.device_status(ws) == 0
        xo, _ = orc.newton_step(s, xo)
    rel = rel_by_degree(x.cpu().numpy(), xo)
    print("ls newton", seed, n, N, "worst rel/eps", float((rel / eps(K)).max()))
    assert float((rel / eps(K)).max()) <= TOL
    # eval_diff shapes with N rows
    f, A = md.eval_diff(sysd, x, ws)
    assert tuple(f.shape) == (s.planes, K, N, d + 1) and tuple(A.shape) == (s.planes, K, d + 1, n, N)
    fo, Ao = orc.eval_diff(s, x.cpu().numpy())
    assert np.array_equal(f.cpu().numpy(), fo) and np.array_equal(A.cpu().numpy(), Ao)


def test_lstsq_refusals(md):
    s = mdgen.config_system(0, 1).augmented([0], [2.0])
    sysd = md.DeviceSystem(s)
    assert sysd.workspace_bytes(md.FLAG_LU) == 0
    assert sysd.workspace_bytes(md.FLAG_OZAKI) == 0
    ws = md.workspace(sysd.workspace_bytes())
    x = md.to_device(s.x0)
    with pytest.raises(md.MdError) as e:
        md.newton_step(sysd, x, ws, flags=md.FLAG_LU)
    assert e.value.code == 1
    with pytest.raises(md.MdError) as e:
        md.newton_step(sysd, x, ws, flags=md.FLAG_OZAKI)
    assert e.value.code == 8
