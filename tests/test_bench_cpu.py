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
    v, t, txt, cores = bench.oracle_sample(pr, level1, cycles, async_m=8)
    assert v > 0 and t > 0 and cores == 1
    m = re.search(r"([\d.]+) s of level-0 work per cycle, ([\d.]+) s per level-1 iteration", txt)
    assert m, txt
    assert "Alg. AsyncMG, m = 8" in txt
    assert f"{cycles} cycles and {level1} level-1 iterations" in txt


def test_cpu_baseline_sample_of_the_multiplicative_cycle():
    pr = workload("sipg2d_p1_16x16").make(0)
    v, t, txt, _ = bench.oracle_sample(pr, 40, 20, async_m=0)
    assert v > 0 and "Alg. 2" in txt


def test_cpu_baseline_all_core_sample_states_its_threads():
    pr = workload("sipg2d_p1_16x16").make(0)
    v, t, txt, cores = bench.oracle_sample(pr, 40, 20, async_m=8, openmp=True)
    assert v > 0 and cores >= 1
    assert txt.startswith(f"{cores} host thread")


def test_traffic_is_null_unless_the_kernel_sources_match():
    assert bench._traffic("no such kernel") == (None, None)
    saved = dict(bench.TRAFFIC)
    try:
        bench.TRAFFIC["k_x"] = (123.0, "0" * 16, ["engine.cu"], "capture note")
        v, note = bench._traffic("k_x")
        assert v is None and "changed" in note
        bench.TRAFFIC["k_x"] = (123.0, bench._sources_sha(["engine.cu"]), ["engine.cu"], "capture note")
        assert bench._traffic("k_x") == (123.0, "capture note")
    finally:
        bench.TRAFFIC.clear()
        bench.TRAFFIC.update(saved)
