"""Host-side checks of the benchmark's CPU-baseline leg (the oracle timed on a bounded
sample; no GPU): it runs on a small workload and extrapolates with its own figures."""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workloads import workload  # noqa: E402


def test_cpu_baseline_sample_extrapolates_level0_and_level1_work():
    pr = workload("sipg2d_p1_16x16").make(0)
    cycles, level1 = 11, 60
    v, t, txt = bench.oracle_sample(pr, level1, cycles, async_m=8)
    assert v > 0 and t > 0
    m = re.search(r"([\d.]+) s of level-0 work per cycle, ([\d.]+) s per level-1 iteration", txt)
    assert m, txt
    assert "Alg. AsyncMG, m = 8" in txt
    assert f"{cycles} cycles and {level1} level-1 iterations" in txt


def test_cpu_baseline_sample_of_the_multiplicative_cycle():
    pr = workload("sipg2d_p1_16x16").make(0)
    v, t, txt = bench.oracle_sample(pr, 40, 20, async_m=0)
    assert v > 0 and "Alg. 2" in txt
