"""The benchmark's FP64-instruction model of the md algorithms against the
counting oracle (the same algorithms): GPU instructions = all binary64 ops
- 3 per TwoSum (done on the GPU as an integer magnitude swap and FastTwoSum)."""
import numpy as np
import pytest

import bench
import mdgen


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 8, 10])
def test_fp64_instruction_model(orc_count, K):
    rng = np.random.default_rng(100 + K)
    x = mdgen.random_md_array(rng, K, 1)[None]
    y = mdgen.random_md_array(rng, K, 1)[None]
    model = bench.fp64_instr_counts(K)
    for op, arg in (("add", y), ("mul", y), ("mul_d", np.array([3.7]))):
        orc_count.count_reset()
        orc_count.md_op(op, K, False, x, arg)
        c = orc_count.counts()
        gpu = c["add"] + c["sub"] + c["mul"] + c["fma"] + c["div"] + c["sqrt"] - 3 * c["twosum"]
        assert gpu == model[op], (K, op, gpu, model[op])


def test_conv_schedule_count(orc_count):
    """Series products of the evaluation schedule, counted by the oracle's
    series-product calls (one md complex mul per term)."""
    s = mdgen.config_system(0, 1)
    orc_count.count_reset()
    orc_count.eval_diff(s, s.x0)
    c = orc_count.counts()
    d = s.degree
    per_conv = (d + 1) * (d + 2) // 2
    # scaling by coefficients: one series mul per output coefficient for every
    # value / partial that is not the unit series
    nconv = bench.conv_schedule_counts(s)
    scal = 0
    for i in range(s.n):
        for _, pairs in s.monomials(i):
            xs = [(v, e) for v, e in pairs if v != s.n]
            at = sum(e for v, e in pairs if v == s.n)
            m = len(xs)
            fch = sum(e - 1 for _, e in xs)
            live = max(d + 1 - at, 0)
            g_unit = (m == 0 and fch == 0)
            scal += 0 if g_unit else live
            for q in range(m):
                d_unit = (m == 1 and fch == 0)
                scal += 0 if d_unit else live
    assert c["series_mul"] == nconv * per_conv + scal
