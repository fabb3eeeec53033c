"""Edge and degenerate cases on the GPU against the oracle: truncation degree
0, one unknown, a polynomial without monomials (singular A_0), constant and
t-only monomials, long series of odd and even degree (the ragged end of the
coefficient pairing), empty inputs, a one-row solve and a one-system batch."""
from fractions import Fraction

import numpy as np
import pytest

import mdgen
from mdcompare import TOL, worst_in_eps

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


def _step_vs_oracle(md, orc, s, steps=2, tol=TOL):
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    x = md.to_device(s.x0)
    xo = s.x0.copy()
    for _ in range(steps):
        md.newton_step(sysd, x, ws)
        assert md.device_status(ws) == 0
        xo, _ = orc.newton_step(s, xo)
    worst = worst_in_eps(x.cpu().numpy(), xo, s.limbs)
    print(s.name, "steps", steps, "worst rel/eps:", worst)
    assert worst <= tol


def _eval_vs_oracle(md, orc, s, x):
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    f, A = md.eval_diff(sysd, md.to_device(x), ws)
    fo, Ao = orc.eval_diff(s, x)
    assert np.array_equal(f.cpu().numpy(), fo) and np.array_equal(A.cpu().numpy(), Ao)


@pytest.mark.parametrize("K,cplx", [(2, True), (4, False)])
def test_degree_zero_is_plain_newton(md, orc, K, cplx):
    s = mdgen.random_system(7, n=4, K=K, cplx=cplx, d=0, monos=4, maxvars=3, maxdeg=3,
                            coef_kind="unit" if cplx else "uniform")
    x0 = s.x0.copy()
    x0[:, 0] *= 1.0 + 1e-3  # start off the solution
    s.x0 = x0
    _step_vs_oracle(md, orc, s, steps=3)


def test_one_unknown(md, orc):
    _step_vs_oracle(md, orc, mdgen.sqrt_system(3, 20, cplx=True), steps=5)


def _tiny(K, d, polys, coefs, csts, x0):
    F = Fraction
    return mdgen._pack(len(x0), K, True, d, polys, [[(F(c), F(0)) for c in cs] for cs in coefs],
                       [(F(c), F(0)) for c in csts], [(F(v), F(0)) for v in x0])


def test_polynomial_without_monomials_is_singular(md, orc):
    """f_1 is a constant: row 1 of A_0 is zero, both sides report a singular A_0."""
    s = _tiny(2, 4, [[[(0, 2)], [(2, 1)]], []], [[1, -1], []], [-1, 3], [1, 0.5])
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    md.newton_step(sysd, md.to_device(s.x0), ws)
    assert md.device_status(ws) == 4
    with pytest.raises(RuntimeError):
        orc.newton_step(s, s.x0)


def test_constant_and_t_only_monomials(md, orc):
    """Monomials without variables (a second constant) and with t alone."""
    polys = [[[], [(2, 3)], [(0, 1), (1, 1)], [(0, 2)]], [[(2, 1)], [(1, 2)], [(0, 1), (2, 2)]]]
    coefs = [[0.25, 2, 1, 0.5], [-1, 1, 0.75]]
    s = _tiny(3, 9, polys, coefs, [-1.75, -1], [1, 1])  # x0 = (1, 1) solves at t = 0, J = [[2, 1], [0, 2]]
    x = s.x0.copy()
    x[:, 0, :, 1:] = np.random.default_rng(3).uniform(-0.5, 0.5, size=x[:, 0, :, 1:].shape)
    _eval_vs_oracle(md, orc, s, x)
    _step_vs_oracle(md, orc, s, steps=2)


@pytest.mark.parametrize("d", [127, 128])
def test_long_series_ragged_pairing(md, orc, d):
    """Coefficient pairs (k, d-k): odd d has none left over, even d a middle one."""
    s = mdgen.random_system(11, n=2, K=2, cplx=True, d=d, monos=3, maxvars=2, maxdeg=3)
    x = s.x0.copy()
    x[:, 0, :, 1:] = np.random.default_rng(d).uniform(-0.5, 0.5, size=x[:, 0, :, 1:].shape) / np.arange(1, d + 1)
    _eval_vs_oracle(md, orc, s, x)


def test_empty_inputs(md):
    import torch

    x = torch.zeros((1, 2, 0), dtype=torch.float64, device="cuda")
    out = md.elementwise("add", 2, False, x, x)
    assert out.numel() == 0
    xs = torch.zeros((1, 2, 0, 5), dtype=torch.float64, device="cuda")
    z = md.series_conv(2, False, xs, xs)
    assert z.numel() == 0


def test_one_row_solve(md, orc):
    K = 4
    rng = np.random.default_rng(5)
    A = np.zeros((2, K, 1, 1, 1))
    A[:, 0] = rng.standard_normal((2, 1, 1, 1))
    b = np.zeros((2, K, 1, 1))
    b[:, 0] = rng.standard_normal((2, 1, 1))
    ws = md.workspace(md.linsolve_workspace_bytes(K, True, 1, 0))
    dx = md.linsolve(K, True, md.to_device(A), md.to_device(b), ws).cpu().numpy()
    want = orc.linsolve(K, True, A, b)
    assert worst_in_eps(dx, want, K) <= TOL


def test_one_system_batch(md):
    """A batch of one system gives the bits of the single-system step."""
    import torch

    s = mdgen.config_system(0, 4)
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    x1 = md.to_device(s.x0)
    md.newton_step(sysd, x1, ws)
    x2 = md.to_device(s.x0)
    bws = md.workspace(md.batched_workspace_bytes([sysd]))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        md.newton_step_batched([sysd], [x2], bws, stream=stream)
    stream.synchronize()
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
