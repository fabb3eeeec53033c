"""Failure detection on the GPU without a fault: the library's one device-side
wait (the batched form's placement gate) is bounded, and when it runs out it
sets a status bit that the host reads as MD_ERR_TIMEOUT; the context stays
usable and the next call's status is clean."""
import time

import pytest

pytestmark = pytest.mark.gpu

MD_OK, MD_ERR_TIMEOUT = 0, 7


@pytest.fixture(scope="module")
def md():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_06607_gb300 import build

    build.build()
    import paper_2012_06607_gb300 as m

    return m


def test_bounded_wait_reports_timeout(md):
    import torch

    ws = md.workspace(4096)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    md.wait_selftest(ws, 1)  # a target nothing reaches
    st = md.device_status(ws)
    waited = time.perf_counter() - t0
    assert st == MD_ERR_TIMEOUT, st
    assert waited < 5.0, waited  # gave up after about 0.1 s
    assert md.device_status(ws) == MD_OK  # the word was cleared by the read


def test_wait_that_ends_leaves_status_clean(md):
    ws = md.workspace(4096)
    md.wait_selftest(ws, 0)
    assert md.device_status(ws) == MD_OK


def test_context_usable_after_timeout(md):
    """A timed-out wait followed by an ordinary computation on the same
    stream: the computation runs and is correct."""
    import torch

    ws = md.workspace(4096)
    md.wait_selftest(ws, 3)
    assert md.device_status(ws) == MD_ERR_TIMEOUT
    x = torch.zeros((1, 2, 64), dtype=torch.float64, device="cuda")
    x[0, 0] = 1.0  # double double 1 (lower limb zero)
    z = md.elementwise("add", 2, False, x, x)
    torch.cuda.synchronize()
    assert float(z[0, 0, 0].item()) == 2.0 and float(z[0, 1].abs().max().item()) == 0.0
