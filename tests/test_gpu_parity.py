"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Elementwise md operations, series products and the evaluation /
differentiation keep the oracle's operation order: they must agree bit for
bit (IEEE equality of every limb).  The block Toeplitz solve runs tree
reductions and an explicit A_0^-1 = R^-1 Q^H, so the solve and the Newton
step are compared within a tolerance: per degree k, the largest difference
over the unknowns is at most 1e3 eps_K times the largest modulus of the
reference's degree-k coefficients, eps_K = 2^(-52 K).  The reference is the
oracle in the same precision, and for whole steps also the oracle run with
more limbs on the same exact inputs (twice the limbs; ten for octo double),
which stands in for the exact step.
"""
import math
import os

import numpy as np
import pytest

import mdgen
from mdcompare import TOL, eps, md_diff, md_value, modulus, rel_by_degree, worst_in_eps

pytestmark = pytest.mark.gpu

KS = [1, 2, 3, 4, 5, 8, 10]


@pytest.fixture(scope="module")
def md():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_06607_gb300 import build

    build.build()
    import paper_2012_06607_gb300 as m

    return m


def _operands(K, P, count, seed):
    rng = np.random.default_rng([K, P, seed])
    x = np.stack([mdgen.random_md_array(rng, K, count, spread=3.0) for _ in range(P)])
    y = np.stack([mdgen.random_md_array(rng, K, count, spread=3.0) for _ in range(P)])
    q = count // 8
    y[:, :, :q] = -x[:, :, :q]  # exact cancellation
    y[:, 1:, q:2 * q] = 0.0  # exact doubles
    x[:, 1:, 2 * q:3 * q] = 0.0
    return x, y


@pytest.mark.parametrize("K", KS)
@pytest.mark.parametrize("cplx", [False, True])
def test_elementwise_bit_exact(md, orc, K, cplx):
    P = 2 if cplx else 1
    x, y = _operands(K, P, 512, 1)
    xd, yd = md.to_device(x), md.to_device(y)
    for op in ("add", "sub", "mul", "div"):
        got = md.elementwise(op, K, cplx, xd, yd).cpu().numpy()
        want = orc.md_op(op, K, cplx, x, y)
        assert np.array_equal(got, want), (op, K, cplx, int((got != want).sum()))
    b = np.random.default_rng(K).standard_normal(512) * 7
    got = md.elementwise("mul_d", K, cplx, xd, md.to_device(b)).cpu().numpy()
    assert np.array_equal(got, orc.md_op("mul_d", K, cplx, x, b))
    if not cplx:
        xa = x * np.sign(x[:, :1, :])
        got = md.elementwise("sqrt", K, False, md.to_device(xa)).cpu().numpy()
        assert np.array_equal(got, orc.md_op("sqrt", K, False, xa)), ("sqrt", K)


@pytest.mark.parametrize("K", [1, 2, 4, 8])
@pytest.mark.parametrize("d", [0, 8, 33, 64])
def test_series_conv_bit_exact(md, orc, K, d):
    rng = np.random.default_rng(K * 100 + d)
    x = rng.standard_normal((2, K, 5, d + 1)) * np.array([2.0 ** (-53 * l) for l in range(K)])[None, :, None, None]
    y = rng.standard_normal((2, K, 5, d + 1)) * np.array([2.0 ** (-53 * l) for l in range(K)])[None, :, None, None]
    got = md.series_conv(K, True, md.to_device(x), md.to_device(y)).cpu().numpy()
    assert np.array_equal(got, orc.series_conv(K, True, x, y))


def _perturbed_x(s, seed, amp=0.5):
    rng = np.random.default_rng(seed)
    x = s.x0.copy()
    x[:, 0, :, 1:] = rng.uniform(-amp, amp, size=x[:, 0, :, 1:].shape)
    if s.limbs > 1:
        x[:, 1, :, 1:] = x[:, 0, :, 1:] * rng.uniform(-1, 1, size=x[:, 0, :, 1:].shape) * 2.0 ** -54
    return x


def _eval_case(md, orc, s, x):
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    f, A = md.eval_diff(sysd, md.to_device(x), ws)
    f_o, A_o = orc.eval_diff(s, x)
    f, A = f.cpu().numpy(), A.cpu().numpy()
    assert np.array_equal(f, f_o), int((f != f_o).sum())
    assert np.array_equal(A, A_o), int((A != A_o).sum())


@pytest.mark.parametrize("K", KS)
@pytest.mark.parametrize("cplx", [False, True])
def test_eval_diff_bit_exact_small(md, orc, K, cplx):
    for seed, (n, d, monos, maxvars, maxdeg) in enumerate([(3, 8, 4, 2, 2), (5, 7, 6, 4, 4), (4, 0, 3, 3, 5),
                                                           (6, 16, 5, 4, 6), (2, 1, 2, 1, 3)]):
        s = mdgen.random_system(seed + 10 * K, n=n, K=K, cplx=cplx, d=d, monos=monos, maxvars=maxvars, maxdeg=maxdeg,
                                coef_kind="unit" if cplx else "uniform", cond_max=1e12)
        _eval_case(md, orc, s, _perturbed_x(s, seed))


def test_eval_diff_bit_exact_examples(md, orc):
    for s in (mdgen.circle_system(2, 8), mdgen.sqrt_system(4, 12), mdgen.config_system(0, 1),
              mdgen.linear_system(1, 4, 2, 5)[0]):
        _eval_case(md, orc, s, _perturbed_x(s, 3, 0.25))


@pytest.mark.parametrize("cfg", [1, 2])
def test_eval_diff_bit_exact_full_size(md, orc, cfg):
    """Full configuration sizes (quad double complex n=64 d=64; octo double real n=128 d=32)."""
    s = mdgen.config_system(cfg, 1)
    _eval_case(md, orc, s, _perturbed_x(s, 5, 0.2))


def _random_linear(K, cplx, n, d, seed, diag=4.0):
    rng = np.random.default_rng(seed)
    P = 2 if cplx else 1
    sc = np.array([2.0 ** (-53 * l) for l in range(K)])
    A = rng.standard_normal((P, K, d + 1, n, n)) * sc[None, :, None, None, None]
    for c in range(n):
        A[0, 0, 0, c, c] += diag
    b = rng.standard_normal((P, K, n, d + 1)) * sc[None, :, None, None]
    return A, b


@pytest.mark.parametrize("K,cplx,n,d", [(2, True, 8, 8), (4, False, 9, 5), (4, True, 16, 12), (8, False, 7, 4),
                                        (1, True, 5, 6), (3, True, 33, 3)])
def test_linsolve_close_to_oracle(md, orc, K, cplx, n, d):
    """Well-conditioned A_0 (diagonally dominant): per degree k,
    max_i |dx_gpu - dx_oracle| <= 1e3 eps_K (k+1) max_i |dx_k|."""
    A, b = _random_linear(K, cplx, n, d, seed=K * 7 + n)
    ws = md.workspace(md.linsolve_workspace_bytes(K, cplx, n, d))
    got = md.linsolve(K, cplx, md.to_device(A), md.to_device(b), ws).cpu().numpy()
    assert md.device_status(ws) == 0
    want = orc.linsolve(K, cplx, A, b)
    rel = rel_by_degree(got, want)
    print("linsolve", K, cplx, n, d, "max rel/eps:", float((rel / eps(K)).max()))
    for k in range(d + 1):
        assert rel[k] <= 1e3 * eps(K) * (k + 1), (k, rel[k] / eps(K))


def test_singular_reported(md):
    K, n, d = 2, 4, 3
    A, b = _random_linear(K, False, n, d, seed=3)
    A[:, :, 0, 1, :] = A[:, :, 0, 0, :]  # two equal columns of A_0
    A[:, :, 0, :, :] = 0.0
    ws = md.workspace(md.linsolve_workspace_bytes(K, False, n, d))
    md.linsolve(K, False, md.to_device(A), md.to_device(b), ws)
    assert md.device_status(ws) == 4
    assert md.device_status(ws) == 0  # cleared after reading


def test_nonfinite_reported(md):
    K, n, d = 2, 4, 3
    A, b = _random_linear(K, False, n, d, seed=4)
    b[0, 0, 1, 2] = np.nan
    ws = md.workspace(md.linsolve_workspace_bytes(K, False, n, d))
    md.linsolve(K, False, md.to_device(A), md.to_device(b), ws)
    assert md.device_status(ws) == 5


def _newton_compare(md, orc, s, steps, tol_factor=TOL):
    """`steps` GPU steps and oracle steps from x0 in the same precision; after
    every step the series agree within tol_factor eps_K per degree, and the
    norm of the last coefficient's update agrees too."""
    import torch

    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    x = md.to_device(s.x0)
    nrm = torch.zeros(2, dtype=torch.float64, device="cuda")
    xo = s.x0.copy()
    worst = 0.0
    for st in range(steps):
        md.newton_step(sysd, x, ws, nrm)
        assert md.device_status(ws) == 0
        xo, nr = orc.newton_step(s, xo)
        rel = rel_by_degree(x.cpu().numpy(), xo)
        worst = max(worst, float((rel / eps(s.limbs)).max()))
        g = nrm.cpu().numpy()
        assert abs(g[0] - nr[0]) <= 1e-6 * max(nr[0], 1e-300) + 1e3 * eps(s.limbs) * max(
            float(np.abs(xo[:, 0]).max()), 1.0)
    print(s.name, "steps", steps, "worst rel err / eps:", worst)
    assert worst <= tol_factor
    return worst


def test_newton_cfg0_four_steps(md, orc):
    _newton_compare(md, orc, mdgen.config_system(0, 1), 4)


def test_newton_examples(md, orc):
    _newton_compare(md, orc, mdgen.circle_system(2, 8), 5)
    _newton_compare(md, orc, mdgen.sqrt_system(4, 16), 5)


@pytest.mark.parametrize("cfg", [1, 2])
def test_newton_full_size_one_step(md, orc, cfg):
    _newton_compare(md, orc, mdgen.config_system(cfg, 1), 1)


def _gpu_steps(md, s, steps):
    import torch

    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    x = md.to_device(s.x0)
    nrm = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(steps):
        md.newton_step(sysd, x, ws, nrm)
        assert md.device_status(ws) == 0
    return x.cpu().numpy()


@pytest.mark.parametrize("cfg,steps,Kref", [(0, 4, 4), (1, 1, 8), (2, 1, 10)])
def test_newton_against_more_limbs(md, orc, cfg, steps, Kref):
    """Whole steps against the oracle with more limbs on the same exact inputs
    (the coefficients, constants and x0 of the K-limb system re-expanded into
    Kref limbs): double double (4 steps, reference quad double), quad double
    (the n = 64, d = 64 step, reference octo double), octo double (the
    n = 128, d = 32 step, reference deca double).  Per degree within
    1e3 eps_K of the reference."""
    s = mdgen.config_system(cfg, 1)
    got = _gpu_steps(md, s, steps)
    ref = s.with_limbs(Kref)
    xr, _ = orc.newton(ref, steps)
    worst = worst_in_eps(got, xr, s.limbs)
    print(s.name, "against", Kref, "limbs: worst rel err / eps_K:", worst)
    assert worst <= TOL


@pytest.mark.parametrize("form", ["plain", "split"])
def test_autotuned_step_equals_default(md, form):
    """MD_FLAG_AUTOTUNE changes how many SMs the factorisation keeps while the
    evaluation runs (one untimed call, then one count per call over the next
    14 calls of a plan, the fastest kept from the 16th on), never the
    result: 18 autotuned steps from x0 give the bits of 18 default steps,
    plain and split-product form, and the tuning has ended by then."""
    import torch

    s = mdgen.config_system(1, 1)
    sysd = md.DeviceSystem(s)
    base = md.FLAG_OZAKI if form == "split" else 0
    outs = []
    for flags in (base, base | md.FLAG_AUTOTUNE):
        ws = md.workspace(sysd.workspace_bytes(flags))
        x = md.to_device(s.x0)
        for _ in range(18):
            md.newton_step(sysd, x, ws, flags=flags)
            torch.cuda.synchronize()
        assert md.device_status(ws) == 0
        outs.append(x.cpu().numpy())
        if flags & md.FLAG_AUTOTUNE:
            assert md.plan_factor_sms(sysd, flags) in (4, 8, 12, 16, 24, 32, 48)
        else:
            assert md.plan_factor_sms(sysd, flags) == 0  # untuned plan: the default count
    assert np.array_equal(outs[0], outs[1])


def test_deterministic(md):
    import torch

    s = mdgen.config_system(0, 2)
    sysd = md.DeviceSystem(s)
    outs = []
    for _ in range(2):
        ws = md.workspace(sysd.workspace_bytes())
        x = md.to_device(s.x0)
        for _ in range(3):
            md.newton_step(sysd, x, ws)
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("cfg", [0, 1])
def test_overlapped_step_equals_serial(md, cfg):
    """The default step factors A_0 on a second stream while the higher
    coefficients are evaluated; MD_FLAG_SERIAL runs every phase in order on the
    caller's stream.  Same bits."""
    import torch

    s = mdgen.config_system(cfg, 1)
    sysd = md.DeviceSystem(s)
    out = []
    for flags in (0, 8):
        ws = md.workspace(sysd.workspace_bytes(flags))
        x = md.to_device(s.x0)
        nrm = torch.zeros(2, dtype=torch.float64, device="cuda")
        for _ in range(2):
            md.newton_step(sysd, x, ws, nrm, flags=flags)
        assert md.device_status(ws) == 0
        out.append((x.cpu().numpy(), nrm.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("K,cplx", [(3, True), (5, False), (10, True), (1, True)])
def test_newton_other_precisions(md, orc, K, cplx):
    """Triple, penta and deca double (and plain double): several Newton steps of
    a random system against the oracle in the same precision."""
    s = mdgen.random_system(40 + K, n=6, K=K, cplx=cplx, d=10, monos=5, maxvars=3, maxdeg=3,
                            coef_kind="unit" if cplx else "uniform", name=f"k{K}")
    _newton_compare(md, orc, s, 4)


def test_newton_octo_double_two_steps(md, orc):
    """Octo double real, n = 128, d = 32: two full steps against the oracle."""
    _newton_compare(md, orc, mdgen.config_system(2, 1), 2)
