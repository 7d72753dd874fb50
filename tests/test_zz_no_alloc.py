"""The no-allocation residual entry point (kcmg_residual_noalloc).

It serves callers that must not allocate device memory: processes whose device memory a
framework's caching allocator already holds, code under a fixed device-memory budget, and
recovery paths after an out-of-memory failure.  Its reduction scratch is a static device
array shared by every call; kcmg_setup looks up its address, so the call itself does no
set-up.  This file is collected last, so that a run stopping at the first failure has
already run every other test.  It must pass alone in a fresh process and after the other
tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2512_08728_gb300 as pkg
from oracle import OracleSolver
from paper_2512_08728_gb300 import kcmg as K
from workloads import make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


@pytest.mark.parametrize("name", ["sipg3d_p2_8cube", "ragged_3d_p2", "sipg2d_p1_16x16"])
def test_residual_noalloc_matches_apply_on_two_calls_in_a_row(name):
    pr = make_problem(3, 2, (6, 6, 2), 2, seed=1) if name == "ragged_3d_p2" else workload(name).make(1)
    s = pkg.KCycleSolver(pr, precision="fp64")
    rng = np.random.default_rng(11)
    dev = torch.device("cuda")
    # every buffer exists before the calls, so device memory can only change by the calls
    xs = [torch.from_numpy(rng.standard_normal(pr.ndof)).to(dev) for _ in range(2)]
    bs = [torch.from_numpy(rng.standard_normal(pr.ndof)).to(dev) for _ in range(2)]
    rs = [torch.empty_like(bs[0]) for _ in range(2)]
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    norms, free_after = [], []
    for call in range(2):
        norms.append(K.kcmg_residual_noalloc(s.ctx, bs[call], xs[call], rs[call]))
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
    # neither call took device memory (the set-up ran inside kcmg_setup)
    assert min(free_after) >= free_before
    orc = OracleSolver.from_problem(pr)
    for call in range(2):
        got = rs[call].cpu().numpy()
        # the existing entry point: y = A x through kcmg_apply, r = b - y
        ref = bs[call].cpu().numpy() - s.apply(0, xs[call].cpu().numpy(), op=0)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        # and the oracle's operator (CPU, FP64)
        ro = bs[call].cpu().numpy() - orc.apply(0, xs[call].cpu().numpy())
        assert np.abs(got - ro).max() <= 1e-13 * np.abs(ro).max()
        assert abs(norms[call] - np.linalg.norm(ro)) <= 1e-12 * np.linalg.norm(ro)
    s.close()


def test_residual_noalloc_rejects_host_buffers():
    pr = workload("sipg2d_p1_16x16").make(0)
    s = pkg.KCycleSolver(pr, precision="fp64")
    with pytest.raises(ValueError):
        K.kcmg_residual_noalloc(s.ctx, np.zeros(pr.ndof), np.zeros(pr.ndof), np.zeros(pr.ndof))
    s.close()
