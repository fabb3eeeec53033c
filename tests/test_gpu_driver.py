"""Newton with degree continuation on the GPU (md_newton_series_run) against
the oracle's driver: the same levels, the same number of steps per level
(the stop decisions are taken on ||dx|| values far from the thresholds), and
the final series within the per-degree tolerance of the step."""
import numpy as np
import pytest

import mdgen
from mdcompare import TOL, eps, worst_in_eps

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


def _run(md, s, x0, degrees, max_iter, tol, too_large, flags=0):
    sysd = md.DeviceSystem(s)
    sc = md.schedule(degrees, max_iter, tol, too_large)
    ws = md.workspace(md.newton_run_workspace_bytes(sysd, sc, flags))
    x = md.to_device(x0)
    rep = md.newton_run(sysd, x, ws, sc, flags)
    return x.cpu().numpy(), rep


def _margin_ok(rep, tol, too_large, factor=1e2):
    """Every decision value is at least `factor` times away from its threshold."""
    for v in rep["dx_norm"]:
        for th in (tol, too_large):
            if th > 0 and v > 0 and 1.0 / factor < v / th < factor:
                return False
    return True


@pytest.mark.parametrize("K,tol", [(2, 1e-28), (4, 1e-58)])
def test_sqrt_ladder(md, orc, K, tol):
    s = mdgen.sqrt_system(K, 16)
    x0 = s.x0.copy()
    x0[0, 0, 0, 1] = 0.5
    xg, rg = _run(md, s, x0, [8, 16], [8, 8], tol, 1.0)
    xo, ro = orc.newton_run(s, [8, 16], [8, 8], tol, 1.0, x0)
    assert rg["iterations"] == ro["iterations"] == [4, 2]
    assert rg["levels_done"] == 2 and rg["converged"]
    assert worst_in_eps(xg, xo, K) <= TOL


def test_too_large_stops(md, orc):
    s = mdgen.sqrt_system(2, 16)
    x0 = s.x0.copy()
    x0[0, 0, 0, 1] = 0.5
    xg, rg = _run(md, s, x0, [8, 16], [2, 8], 1e-28, 1e-6)
    xo, ro = orc.newton_run(s, [8, 16], [2, 8], 1e-28, 1e-6, x0)
    assert rg["levels_done"] == ro["levels_done"] == 1 and not rg["converged"]
    assert rg["dx_norm"][0] == pytest.approx(ro["dx_norm"][0], rel=1e-12)
    assert np.array_equal(xg[..., 9:], x0[..., 9:])


@pytest.mark.parametrize("seed", [1, 2, 6])
def test_random_system_ladder(md, orc, seed):
    """dd complex n=3, degrees 2 -> 4 -> 8 (the paper's 8/8/12-style limits).
    The seeds are chosen so that every stop decision of the oracle's run is at
    least three decades away from its threshold (asserted): rounding
    differences between the GPU and the oracle cannot flip one."""
    s = mdgen.config_system(0, seed)
    degrees, max_iter, tol, tl = [2, 4, 8], [6, 6, 8], 1e-26, 1e3
    xo, ro = orc.newton_run(s, degrees, max_iter, tol, tl)
    assert _margin_ok(ro, tol, tl, 1e3), ro["dx_norm"]
    xg, rg = _run(md, s, s.x0, degrees, max_iter, tol, tl)
    assert rg["levels_done"] == ro["levels_done"]
    assert rg["iterations"] == ro["iterations"]
    assert rg["converged"] == ro["converged"]
    worst = worst_in_eps(xg, xo, 2)
    print("driver seed", seed, "worst rel/eps:", worst)
    assert worst <= TOL


def test_one_level_equals_steps(md):
    """One level without a stop is the plain step repeated, bit for bit."""
    import torch

    s = mdgen.config_system(0, 3)
    xg, rg = _run(md, s, s.x0, [s.degree], [3], 0.0, 1e300)
    sysd = md.DeviceSystem(s)
    ws = md.workspace(sysd.workspace_bytes())
    x = md.to_device(s.x0)
    nrm = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(3):
        md.newton_step(sysd, x, ws, nrm)
    assert np.array_equal(xg, x.cpu().numpy())
    assert rg["iterations"] == [3] and rg["dx_norm"][0] == float(nrm[0].item())
