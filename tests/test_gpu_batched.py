"""Batched form: many systems of uneven size and precision in one persistent
launch per precision class.  Each system must get exactly the bits of the
single-system step (same per-item bodies and reduction trees), with and
without the autotuner and the CUDA graph, and every system of a mixed batch
of full-width inputs must agree with the oracle's Newton step within the
per-degree tolerance (1e3 eps_K)."""
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


def _mixed_systems():
    rng = np.random.default_rng(77)
    out = []
    for b in range(20):
        n = int(rng.integers(3, 11))
        d = int(rng.integers(2, 10))
        K = [2, 4, 3, 1][b % 4]
        out.append(mdgen.small_system_fast(rng, n, d, K, monos=n, name=f"mix{b}"))
    out.append(mdgen.config_system(0, 2))  # the n = 3 double-double configuration
    out.append(mdgen.random_system(9, n=5, K=2, cplx=False, d=6, monos=4, maxvars=3, maxdeg=3, coef_kind="uniform"))
    out.append(mdgen.circle_system(4, 8))
    return out


def _single_steps(md, systems, steps):
    import torch

    xs, norms = [], []
    for s in systems:
        sd = md.DeviceSystem(s)
        ws = md.workspace(sd.workspace_bytes())
        x = md.to_device(s.x0)
        nrm = torch.zeros(2, dtype=torch.float64, device="cuda")
        for _ in range(steps):
            md.newton_step(sd, x, ws, nrm)
        assert md.device_status(ws) == 0
        xs.append(x.cpu().numpy())
        norms.append(nrm.cpu().numpy())
    return xs, norms


def _batched_steps(md, systems, steps, flags=0, stream=None):
    import torch

    sds = [md.DeviceSystem(s) for s in systems]
    ws = md.workspace(md.batched_workspace_bytes(sds, flags))
    xs = [md.to_device(s.x0) for s in systems]
    nrm = torch.zeros((len(systems), 2), dtype=torch.float64, device="cuda")
    times = torch.zeros((len(systems), 2), dtype=torch.int64, device="cuda")
    for _ in range(steps):
        md.newton_step_batched(sds, xs, ws, nrm, times, flags=flags, stream=stream)
    torch.cuda.synchronize()
    assert md.device_status(ws) == 0
    return [x.cpu().numpy() for x in xs], nrm.cpu().numpy(), times.cpu().numpy()


def test_batched_equals_single_system_steps(md):
    systems = _mixed_systems()
    want_x, want_n = _single_steps(md, systems, 2)
    got_x, got_n, times = _batched_steps(md, systems, 2)
    for i, s in enumerate(systems):
        assert np.array_equal(got_x[i], want_x[i]), (i, s.name, s.limbs, s.n, s.degree)
        assert np.array_equal(got_n[i], want_n[i]), (i, s.name)
    assert (times[:, 1] >= times[:, 0]).all() and (times[:, 0] > 0).all()


def test_batched_autotune_and_graph(md):
    import torch

    systems = _mixed_systems()[:12]
    ref_x, ref_n, _ = _batched_steps(md, systems, 3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        got_x, got_n, _ = _batched_steps(md, systems, 3, flags=md.FLAG_AUTOTUNE | md.FLAG_GRAPH, stream=stream)
    for i in range(len(systems)):
        assert np.array_equal(got_x[i], ref_x[i]), i
        assert np.array_equal(got_n[i], ref_n[i]), i


def test_batched_rejects_large_limbs(md):
    s = mdgen.config_system(0, 1).with_limbs(8)
    sd = md.DeviceSystem(s)
    ws = md.workspace(1 << 20)
    x = md.to_device(s.x0)
    with pytest.raises(md.MdError) as e:
        md.newton_step_batched([sd], [x], ws)
    assert e.value.code == 8  # MD_ERR_UNSUPPORTED


def _skewed_systems():
    """A few systems much larger than the rest, so that the most expensive ones
    get a whole SM while the rest of the same precision class share SMs."""
    rng = np.random.default_rng(91)
    out = [mdgen.small_system_fast(rng, 24, 12, 2, monos=24, name="big0"),
           mdgen.small_system_fast(rng, 20, 10, 2, monos=20, name="big1")]
    out += [mdgen.small_system_fast(rng, 8, 6, 2, monos=8, name=f"mid{b}") for b in range(4)]
    out += [mdgen.small_system_fast(rng, int(rng.integers(2, 5)), int(rng.integers(1, 4)), 2, monos=4,
                                    name=f"tiny{b}") for b in range(300)]
    out += [mdgen.small_system_fast(rng, 4, 3, 4, monos=4, name=f"qd{b}") for b in range(40)]
    return out


def test_batched_whole_sm_split_equals_shared_and_single(md):
    import torch

    systems = _skewed_systems()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        split_x, split_n, times = _batched_steps(md, systems, 2, flags=md.FLAG_AUTOTUNE | md.FLAG_GRAPH, stream=stream)
        shared_x, shared_n, _ = _batched_steps(md, systems, 2, flags=md.FLAG_SERIAL, stream=stream)
    pick = [0, 1, 2, 5, 6, 100, 305, len(systems) - 1]
    want_x, want_n = _single_steps(md, [systems[i] for i in pick], 2)
    for i in range(len(systems)):
        assert np.array_equal(split_x[i], shared_x[i]), (i, systems[i].name)
        assert np.array_equal(split_n[i], shared_n[i]), (i, systems[i].name)
    for j, i in enumerate(pick):
        assert np.array_equal(split_x[i], want_x[j]), (i, systems[i].name)
        assert np.array_equal(split_n[i], want_n[j]), (i, systems[i].name)
    assert (times[:, 1] >= times[:, 0]).all() and (times[:, 0] > 0).all()


def test_batched_phase_times(md):
    """MD_FLAG_PHASE_TIMES: ten ordered stamps per system, results unchanged."""
    import torch

    systems = _mixed_systems()[:10]
    ref_x, ref_n, _ = _batched_steps(md, systems, 1)
    sds = [md.DeviceSystem(s) for s in systems]
    ws = md.workspace(md.batched_workspace_bytes(sds))
    xs = [md.to_device(s.x0) for s in systems]
    nrm = torch.zeros((len(systems), 2), dtype=torch.float64, device="cuda")
    times = torch.zeros((len(systems), md.PHASE_STAMPS), dtype=torch.int64, device="cuda")
    md.newton_step_batched(sds, xs, ws, nrm, times, flags=md.FLAG_PHASE_TIMES)
    torch.cuda.synchronize()
    assert md.device_status(ws) == 0
    t = times.cpu().numpy()
    assert (t[:, 0] > 0).all() and (np.diff(t, axis=1) >= 0).all()
    for i in range(len(systems)):
        assert np.array_equal(xs[i].cpu().numpy(), ref_x[i]), i
        assert np.array_equal(nrm.cpu().numpy()[i], ref_n[i]), i


def test_batched_fresh_buffers_every_call(md):
    """A caller that passes new x buffers on every call gets a new plan each
    time; the plan cache drops the least recently used ones (pinned images and
    graphs freed after a device synchronisation) and every result stays the
    same."""
    import torch

    systems = _mixed_systems()[:6]
    ref_x, ref_n, _ = _batched_steps(md, systems, 1)
    sds = [md.DeviceSystem(s) for s in systems]
    ws = md.workspace(md.batched_workspace_bytes(sds))
    stream = torch.cuda.Stream()
    for it in range(24):  # more than the cache holds
        xs = [md.to_device(s.x0) for s in systems]
        nrm = torch.zeros((len(systems), 2), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            md.newton_step_batched(sds, xs, ws, nrm, None, flags=md.FLAG_GRAPH if it % 2 else 0, stream=stream)
        stream.synchronize()
        for i in range(len(systems)):
            assert np.array_equal(xs[i].cpu().numpy(), ref_x[i]), (it, i)
            assert np.array_equal(nrm.cpu().numpy()[i], ref_n[i]), (it, i)
    assert md.device_status(ws) == 0


def _full_width_batch():
    """Double double and quad double complex systems of uneven n and d built by
    mdgen.random_system: unit-modulus coefficients and x0 whose every limb is
    in use, constants fixed exactly so that x0 solves at t = 0."""
    out = []
    specs = [(2, 8, 8), (4, 6, 12), (2, 13, 5), (4, 9, 9), (2, 16, 16), (4, 3, 20), (2, 24, 10), (4, 20, 6),
             (2, 5, 31), (4, 12, 17), (2, 1, 9), (4, 32, 8)]
    for i, (K, n, d) in enumerate(specs):
        out.append(mdgen.random_system(300 + i, n=n, K=K, cplx=True, d=d, monos=max(n, 3), minvars=1, maxvars=2,
                                       maxdeg=3, coef_kind="unit", name=f"fw{i}"))
    return out


def _oracle_steps(orc, s, steps):
    xo = s.x0.copy()
    norms = []
    for _ in range(steps):
        xo, nr = orc.newton_step(s, xo)
        norms.append(nr)
    return xo, norms


def _assert_batch_matches_oracle(orc, systems, got_x, got_n, steps):
    worst_all = 0.0
    for i, s in enumerate(systems):
        xo, norms = _oracle_steps(orc, s, steps)
        worst = worst_in_eps(got_x[i], xo, s.limbs)
        worst_all = max(worst_all, worst)
        assert worst <= TOL, (i, s.name, s.limbs, s.n, s.degree, worst)
        # the norm of the last coefficient's update, within the same tolerance
        scale = max(float(np.abs(xo[:, 0]).max()), 1.0)
        assert abs(got_n[i][0] - norms[-1][0]) <= 1e-6 * norms[-1][0] + TOL * 2.0 ** (-52 * s.limbs) * scale, (
            i, got_n[i][0], norms[-1][0])
    return worst_all


def test_batched_against_oracle_full_width(md, orc):
    """One mixed batch (dd and qd, n from 1 to 32, d from 5 to 31), two Newton
    steps, every system against two oracle steps."""
    systems = _full_width_batch()
    got_x, got_n, _ = _batched_steps(md, systems, 2)
    worst = _assert_batch_matches_oracle(orc, systems, got_x, got_n, 2)
    print("batched vs oracle, full-width mixed batch: worst rel/eps", worst)


def _skewed_full_width():
    """A few large double-double systems among many small ones and some quad
    double ones, all full width: the autotuner then runs the small ones
    several CTAs per SM and gives the largest whole SMs."""
    out = [mdgen.random_system(400, n=24, K=2, cplx=True, d=12, monos=24, maxvars=2, maxdeg=3, name="big0"),
           mdgen.random_system(401, n=20, K=2, cplx=True, d=10, monos=20, maxvars=2, maxdeg=3, name="big1")]
    out += [mdgen.random_system(410 + b, n=8, K=2, cplx=True, d=6, monos=8, maxvars=2, maxdeg=3, name=f"mid{b}")
            for b in range(4)]
    rng = np.random.default_rng(5)
    out += [mdgen.random_system(500 + b, n=int(rng.integers(2, 5)), K=2, cplx=True, d=int(rng.integers(1, 4)),
                                monos=4, maxvars=2, maxdeg=3, name=f"tiny{b}") for b in range(300)]
    out += [mdgen.random_system(900 + b, n=4, K=4, cplx=True, d=3, monos=4, maxvars=2, maxdeg=3, name=f"qd{b}")
            for b in range(40)]
    return out


def test_batched_skewed_against_oracle(md, orc):
    """The skewed batch through the autotuner and the graph (whole-SM CTAs for
    the largest systems when the tuner shares SMs), every system against the
    oracle."""
    import torch

    systems = _skewed_full_width()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        got_x, got_n, _ = _batched_steps(md, systems, 2, flags=md.FLAG_AUTOTUNE | md.FLAG_GRAPH, stream=stream)
    worst = _assert_batch_matches_oracle(orc, systems, got_x, got_n, 2)
    print("batched vs oracle, skewed full-width batch: worst rel/eps", worst)


def test_batched_split_products_against_oracle(md, orc):
    """The split-product form in the batched step (series products on 32-bit
    word slices, MD_FLAG_OZAKI): the full-width mixed batch (two steps) and,
    through the autotuner and the graph, the skewed one (one step), against
    the oracle.  The skewed batch takes one step because its largest system
    (n = 24, d = 12, double double) magnifies the first step's rounding in the
    second: there the double-double oracle itself lies 1.4e3 eps_2 from the
    quad double one, and only the plain form, which has the oracle's bits,
    meets 1e3 eps_2 after two steps."""
    import torch

    systems = _full_width_batch()
    got_x, got_n, _ = _batched_steps(md, systems, 2, flags=md.FLAG_OZAKI)
    worst = _assert_batch_matches_oracle(orc, systems, got_x, got_n, 2)
    print("batched split form vs oracle, full-width mixed batch: worst rel/eps", worst)
    systems = _skewed_full_width()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        got_x, got_n, _ = _batched_steps(md, systems, 1, flags=md.FLAG_OZAKI | md.FLAG_AUTOTUNE | md.FLAG_GRAPH,
                                         stream=stream)
    worst = _assert_batch_matches_oracle(orc, systems, got_x, got_n, 1)
    print("batched split form vs oracle, skewed batch: worst rel/eps", worst)


def test_batched_graph_switches_form(md):
    """The same systems, buffers and stream called with and without
    MD_FLAG_OZAKI under MD_FLAG_GRAPH, alternating: each form replays its own
    plan and graph, so the plain calls keep the bits of the uncaptured plain
    step and the split calls differ from them within the tolerance."""
    import torch

    systems = _mixed_systems()
    ref_x, _, _ = _batched_steps(md, systems, 1)
    sds = [md.DeviceSystem(s) for s in systems]
    flags_all = md.FLAG_GRAPH | md.FLAG_OZAKI
    ws = md.workspace(md.batched_workspace_bytes(sds, flags_all))
    xs = [md.to_device(s.x0) for s in systems]
    x0 = [md.to_device(s.x0) for s in systems]
    nrm = torch.zeros((len(systems), 2), dtype=torch.float64, device="cuda")
    times = torch.zeros((len(systems), 2), dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    split_differs = False
    with torch.cuda.stream(stream):
        for flags in (md.FLAG_GRAPH, flags_all, md.FLAG_GRAPH, flags_all):
            for x, x_init in zip(xs, x0):
                x.copy_(x_init)
            md.newton_step_batched(sds, xs, ws, nrm, times, flags=flags, stream=stream)
            stream.synchronize()
            assert md.device_status(ws) == 0
            for i, s in enumerate(systems):
                got = xs[i].cpu().numpy()
                if flags & md.FLAG_OZAKI:
                    split_differs |= not np.array_equal(got, ref_x[i])
                    assert worst_in_eps(got, ref_x[i], s.limbs) <= TOL, (flags, i)
                else:
                    assert np.array_equal(got, ref_x[i]), (flags, i)
    assert split_differs  # the split form ran, not the captured plain graph
