"""Host logic of bench.py that needs no GPU: the workloads behind --config and
the FP64 instruction model's scaling."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_metric_and_workload():
    import bench

    m, w = bench.metric_and_workload(1, 1)
    assert m == bench.METRIC and "seed 1" in w and "quad double complex" in w
    m, w = bench.metric_and_workload(2, 3)
    assert "od, n=128, d=32" in m and "octo double real" in w and "seed 3" in w
    m, w = bench.metric_and_workload(0, 2)
    assert "dd, n=3, d=8" in m and "seed 2" in w
    with pytest.raises(KeyError):
        bench.metric_and_workload(7, 1)


def test_fp64_model_scales_with_degree_and_limbs():
    import bench
    import mdgen

    s = mdgen.config_system(0, 1)
    m2 = bench.step_fp64_model(s)
    m4 = bench.step_fp64_model(s.with_limbs(4))
    assert m4["conv"] > 3 * m2["conv"] and m4["total"] > 3 * m2["total"]
    assert m2["total"] == pytest.approx(sum(v for k, v in m2.items() if k != "total"))


def test_run_form_uses_the_papers_octo_double_schedule():
    """--form run follows Table 2's octo double row (Section 6): the truncation
    degrees, the iteration counts as per-level limits, and the quoted seconds
    (tests/golden/table2_octo_double.txt)."""
    import bench

    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "table2_octo_double.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    assert tuple(r[0] for r in rows) == bench.RUN_DEGREES
    assert tuple(r[1] for r in rows) == bench.RUN_MAX_ITER
    assert {r[0]: r[2] for r in rows} == bench.PAPER_TABLE2_OD_SECONDS
