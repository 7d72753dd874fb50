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


def _max_over_ranks_rank(rank, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        # rank r timed 1.5 + r seconds: both see the slower rank's time
        q.put((rank, bench._max_over_ranks(1.5 + rank, 2, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    """The multi-rank timing step of the bench (the maximum of the ranks' times) with two
    gloo ranks on the CPU; one rank returns its own value without a process group."""
    import multiprocessing as mp
    import socket
    assert bench._max_over_ranks(3.25, 1, "cpu") == 3.25
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_max_over_ranks_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2.5), (1, 2.5)]
