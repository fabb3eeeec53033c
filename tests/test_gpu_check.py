"""Bounds mode (MD_FLAG_CHECK): the host checks of every plan table index and
of the workspace layout pass for the workloads, and the results are the same
bits as without the checks."""
import numpy as np
import pytest

import mdgen

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


@pytest.mark.parametrize("cfg", [0, 1, 2])
def test_step_with_checks_same_bits(md, cfg):
    import torch

    s = mdgen.config_system(cfg, 1)
    sd = md.DeviceSystem(s)
    out = []
    for flags in (0, md.FLAG_CHECK):
        ws = md.workspace(sd.workspace_bytes())
        x = md.to_device(s.x0)
        nrm = torch.zeros(2, dtype=torch.float64, device="cuda")
        md.newton_step(sd, x, ws, nrm, flags=flags)
        assert md.device_status(ws) == 0
        out.append((x.cpu().numpy(), nrm.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_batched_with_checks_same_bits(md):
    import torch

    rng = np.random.default_rng(5)
    systems = [mdgen.small_system_fast(rng, int(rng.integers(3, 9)), int(rng.integers(2, 8)), [2, 4][b % 2],
                                       monos=4) for b in range(12)]
    sds = [md.DeviceSystem(s) for s in systems]
    res = []
    for flags in (0, md.FLAG_CHECK):
        ws = md.workspace(md.batched_workspace_bytes(sds))
        xs = [md.to_device(s.x0) for s in systems]
        nrm = torch.zeros((len(systems), 2), dtype=torch.float64, device="cuda")
        md.newton_step_batched(sds, xs, ws, nrm, None, flags=flags)
        torch.cuda.synchronize()
        assert md.device_status(ws) == 0
        res.append(([x.cpu().numpy() for x in xs], nrm.cpu().numpy()))
    for i in range(len(systems)):
        assert np.array_equal(res[0][0][i], res[1][0][i]), i
    assert np.array_equal(res[0][1], res[1][1])
