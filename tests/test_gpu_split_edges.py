"""Edge and degenerate cases of the split-product form (MD_FLAG_OZAKI) on the
GPU, from three limbs on, where its series products, accumulation and the
update run on word and byte slices: truncation degree 0, one unknown, long
series of odd and even degree (the ragged end of the coefficient pairing)
against the oracle at 1e3 eps_K; a singular A_0 and a non-finite input
reported as in the plain form; the bounds mode with the same bits."""
from fractions import Fraction

import numpy as np
import pytest

import mdgen
from mdcompare import TOL, worst_in_eps

pytestmark = pytest.mark.gpu

OZAKI, CHECK = 0x1, 0x40


@pytest.fixture(scope="module")
def md():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_06607_gb300 import build

    build.build()
    import paper_2012_06607_gb300 as m

    return m


def _split_steps(md, s, steps, flags=OZAKI):
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes(flags))
    x = md.to_device(s.x0)
    statuses = []
    for _ in range(steps):
        md.newton_step(sysd, x, ws, flags=flags)
        statuses.append(md.device_status(ws))
    return x.cpu().numpy(), statuses


def _vs_oracle(md, orc, s, steps):
    got, statuses = _split_steps(md, s, steps)
    assert statuses == [0] * steps
    xo = s.x0.copy()
    for _ in range(steps):
        xo, _ = orc.newton_step(s, xo)
    worst = worst_in_eps(got, xo, s.limbs)
    print(s.name, "split form, steps", steps, "worst rel/eps:", worst)
    assert worst <= TOL


@pytest.mark.parametrize("K,cplx", [(3, True), (4, False)])
def test_split_degree_zero_is_plain_newton(md, orc, K, cplx):
    s = mdgen.random_system(7, n=4, K=K, cplx=cplx, d=0, monos=4, maxvars=3, maxdeg=3,
                            coef_kind="unit" if cplx else "uniform")
    x0 = s.x0.copy()
    x0[:, 0] *= 1.0 + 1e-3  # start off the solution
    s.x0 = x0
    _vs_oracle(md, orc, s, 3)


@pytest.mark.parametrize("K", [3, 5])
def test_split_one_unknown(md, orc, K):
    _vs_oracle(md, orc, mdgen.sqrt_system(K, 20, cplx=True), 5)


@pytest.mark.parametrize("d", [31, 32])
def test_split_ragged_pairing(md, orc, d):
    """Coefficient pairs (k, d-k) in the fixed-point products: odd d has none
    left over, even d a middle coefficient alone."""
    s = mdgen.random_system(11, n=3, K=4, cplx=True, d=d, monos=3, maxvars=2, maxdeg=3)
    _vs_oracle(md, orc, s, 2)


def test_split_singular_a0_reported(md):
    """A polynomial without monomials: row 1 of A_0 is zero, and the split form
    reports the singular A_0 as the plain form does."""
    F = Fraction
    polys = [[[(0, 2)], [(2, 1)]], []]
    s = mdgen._pack(2, 4, True, 4, polys, [[(F(1), F(0)), (F(-1), F(0))], []], [(F(-1), F(0)), (F(3), F(0))],
                    [(F(1), F(0)), (F(0.5), F(0))])
    got = {}
    for flags in (0, OZAKI):
        _, statuses = _split_steps(md, s, 1, flags=flags)
        got[flags] = statuses[0]
    # MD_ERR_SINGULAR, or MD_ERR_NONFINITE where the singular column's NaN
    # reached dx first: the same in both forms
    assert got[OZAKI] == got[0] and got[0] in (4, 5), got


def test_split_nonfinite_input_reported(md):
    """A NaN limb in x: the split form's fixed-point paths and its 8-bit-slice
    update (a row or vector with a non-finite limb marks its outputs NaN)
    carry it through to dx and report the same status as the plain form."""
    s = mdgen.random_system(3, n=5, K=4, cplx=True, d=6, monos=5, maxvars=2, maxdeg=3)
    x0 = s.x0.copy()
    x0[0, 1, 2, 3] = np.nan
    s.x0 = x0
    got = {}
    for flags in (0, OZAKI):
        x, statuses = _split_steps(md, s, 1, flags=flags)
        got[flags] = statuses[0]
        assert not np.isfinite(x).all(), flags
    assert got[OZAKI] == got[0] != 0


def test_split_bounds_mode_same_bits(md):
    """MD_FLAG_CHECK (the host checks of the plan and of the workspace layout,
    the fixed-point copies included) changes no bit of the split form."""
    s = mdgen.config_system(1, 1)
    a, sa = _split_steps(md, s, 2)
    b, sb = _split_steps(md, s, 2, flags=OZAKI | CHECK)
    assert sa == sb == [0, 0]
    assert np.array_equal(a, b)
