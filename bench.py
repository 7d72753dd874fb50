#!/usr/bin/env python3
"""DOFs solved per second to a relative residual of 1e-10 by the orthonormalization
multigrid (Alg. 1 after every correction, block-Jacobi smoother, level-local criteria of
Sec. 4.2) on one GB300.

Workload: 3-D SIPG p=2 (Np = 10) on 64^3 cells = 2,621,440 DOFs, coefficient 1000 inside a
ball of radius 0.3 and 1 outside, zero Dirichlet, b iid U[-1,1] from the seed, 5-level
2x2x2 agglomeration hierarchy, solved in FP64.  The headline runs level 0 as the paper's
task-parallel cycle (Alg. AsyncMG, fixed smoother count): the coarse path on a second
stream, the smoother path beside it, one join per cycle; levels >= 1 are K-cycles (Alg. 2).
Beside it: the multiplicative K-cycle of Alg. 2 on level 0, and the mixed forms (FP32
smoother sweeps, optionally BF16-stored block inverses, FP64 residual minimisation).

One step = one complete solve from x0 = 0 with inputs resident in device memory.  The
operator (1.47 GB) is larger than the 129 MB L2, so no flush is needed between steps.
Under torchrun every rank solves its own replica (seed = rank): the method has no
data-parallel split on one node here ("replicas only"), so there is no collective.

Timed work: the headline solve at --steps solves after --warmup; each extra form (the
multiplicative cycle, the mixed forms) one solve after its capture; the end-to-end leg
through host buffers at most three solves.  Setup (hierarchy, inverses, graph capture) is
timed separately and reported as setup_s.

--impl reference times the CPU oracle (oracle/, plain C; its OpenMP build on all host
cores) on the same workload: each step is a bounded sample (the first level-0 cycle and
one level-1 visit), extrapolated to the full solve by the level-0 cycle and level-1
iteration counts of the GPU solve.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "sipg3d_p2_64cube"
RTOL = 1e-10
LMAX = 400         # level-0 restart length of the benchmarked configuration
MAXITER = 4000
METRIC = "DOFs solved/s to 1e-10 rel. residual, mixed vs FP64; % of HBM roofline"
UNIT = "DOF/s"
# Level-0 cycle of the headline solve: Alg. AsyncMG (the paper's task-parallel cycle) with
# HEADLINE_ASYNC_M smoother + RM steps per cycle beside the coarse path; the multiplicative
# K-cycle of Alg. 2 (async 0) and the mixed forms are reported beside it.
HEADLINE_ASYNC_M = 12
# the additive Schwarz smoother of the Schwarz forms (Alg. AS on 2^d-cell patches) and the
# level-0 cycle each Schwarz form runs (best mean over seeds 0/1/2 on GB300)
AS_OMEGA = 0.5
AS_SWEEPS = 2
AS_ASYNC_M_FP64 = 16
AS_ASYNC_M_MIXED = 12
# the stretched p = 3 workload of the mixed-precision configuration
STRETCHED = "sipg3d_p3_48cube_zstretch"
STRETCHED_ASYNC_M = 12
# Level-0 cycles and level-1 iterations of the headline FP64 solve of this workload (seed 0,
# LMAX = 400, m = 12), measured on GB300; the reference arm (a separate process)
# extrapolates its bounded sample with them.
GPU_LEVEL1_ITERS_FP64 = 1064
GPU_CYCLES_FP64 = 54


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 FMA peak of GB300 from its unit counts and clock: 152 SMs x 2 FP64 FMA per clock
# per SM x 2 flop x 2.07 GHz = 1.259 TFLOP/s (NVIDIA's nominal 1.25 TFLOP/s).  Kernels
# that do one FP64 FMA per 8-byte element they read are bound by it at 5.03 TB/s, below
# the measured HBM copy bandwidth.
GB300_SMS = 152
FP64_FMA_PER_CLK_PER_SM = 2
SM_MAX_GHZ = 2.07
FP64_TFLOPS = GB300_SMS * FP64_FMA_PER_CLK_PER_SM * 2 * SM_MAX_GHZ / 1e3
FP64_PEAK_NOTE = ("FP64 FMA peak from unit counts and clock: 152 SMs x 2 FMA/clk x 2 flop x "
                  "2.07 GHz = %.3f TFLOP/s, i.e. %.0f GB/s of 8-byte operands at one FMA each"
                  % (FP64_TFLOPS, FP64_TFLOPS * 1e3 / 2 * 8))

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels the bench
# reports, from one ncu capture each, as bytes per unit of work (k_gram_update: per
# (basis column + 2.5) x DOF, the unit its algorithmic bytes (2 l + 5) N 8 count), keyed by
# kernel; valid only while the kernel's sources hash to the recorded value (otherwise the
# line reports null).
TRAFFIC = {
    "k_gram_update": (3567589888.0 / ((2 * 199 + 5) * 1105920), "41bfa758cbb3ac94",
                      ["kernels.cu", "kcmg_internal.h", "reduce.cuh"],
                      "ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of one level-0 "
                      "launch on 48^3 p=2 with 199 basis vectors: 3.568 GB per launch, scaled to "
                      "this launch by (2 l + 5) N"),
}


def _sources_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2512_08728_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel):
    t = TRAFFIC.get(kernel)
    if not t:
        return None, None
    per_launch, sha, files, note = t
    if _sources_sha(files) != sha:
        return None, "kernel changed since the capture (" + note + ")"
    return per_launch, note


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _max_over_ranks(v, ws, dev):
    """The largest v over the ranks of the job (v itself at one rank).  The timed region
    of a multi-rank job ends when its slowest rank ends, so rates divide by this maximum."""
    if ws <= 1:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_sample(pr, level1_total, cycles_total, async_m=None, openmp=False):
    """Time the CPU oracle on a bounded sample of the headline solve and extrapolate.

    The sample is the first level-0 cycle (the same cycle as the headline) plus one level-1
    visit on its own (the level-1 operator as the finest level of a hierarchy one level
    shorter, stopped by the level-1 criteria).  The level-1 visit gives the cost of a
    level-1 iteration (with everything below it); the rest of the first cycle is the
    cost of the level-0 work of a cycle.  The full solve is
    cycles_total x (level-0 cost) + level1_total x (level-1 cost).  The level-0 cost of
    the first cycle is a lower bound for later cycles (their Gram work grows with the
    basis), so the estimate errs towards a faster oracle.
    openmp: the OpenMP build of the oracle on all host cores (its parallel loops give
    bitwise the serial results).
    Returns (dof_per_s, seconds_of_the_sample, text, cores)."""
    import oracle
    am = HEADLINE_ASYNC_M if async_m is None else async_m
    cores = oracle.threads(0) if openmp else 1
    t0 = time.perf_counter()
    orc = oracle.OracleSolver.from_problem(pr, lmax=LMAX, async_smooth=am, openmp=openmp)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    x, info = orc.solve(pr.b, rtol=RTOL, maxiter=1)
    t_cycle = time.perf_counter() - t0
    l1 = int(info["level_iters"][1])
    # one level-1 visit on its own
    rt, mi = oracle.default_level_criteria(pr.nlevels)
    n1 = [v // 2 for v in pr.n]
    o1 = oracle.OracleSolver(pr.d, pr.np_, n1, pr.nlevels - 1, orc.blocks(1), pr.prolong,
                             lvl_rtol=rt[1:], lvl_maxit=mi[1:], openmp=openmp)
    b1 = orc.restrict(0, pr.b)
    t0 = time.perf_counter()
    _, i1 = o1.solve(b1, rtol=float(rt[1]), maxiter=int(mi[1]))
    t_visit = time.perf_counter() - t0
    k1 = max(1, int(i1["iters"]))
    c1 = t_visit / k1
    c0 = max(t_cycle - l1 * c1, 0.0)
    t_full = cycles_total * c0 + level1_total * c1
    cyc = f"Alg. AsyncMG, m = {am}" if am > 0 else "Alg. 2"
    txt = (f"{cores} host thread{'s' if cores > 1 else ''}: "
           f"first level-0 cycle of the solve ({cyc}; {l1} level-1 iterations) "
           f"in {t_cycle:.2f} s and one level-1 visit on its own ({k1} iterations) in "
           f"{t_visit:.2f} s (setup {t_setup:.1f} s, not counted): {c0:.2f} s of level-0 work "
           f"per cycle, {c1:.3f} s per level-1 iteration, extrapolated to the {cycles_total} "
           f"cycles and {level1_total} level-1 iterations of the full solve: {t_full:.0f} s")
    del orc, o1, x
    return pr.ndof / t_full, t_cycle + t_visit, txt, cores


def run_reference(args, ws, rank):
    from workloads import workload
    if rank != 0:
        return
    pr = workload(WORKLOAD).make(0)
    vals = []
    txt = ""
    cores = 1
    for k in range(args.warmup + args.steps):
        v, t, txt, cores = oracle_sample(pr, GPU_LEVEL1_ITERS_FP64, GPU_CYCLES_FP64, openmp=True)
        if k >= args.warmup:
            vals.append((v, t))
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(t for _, t in vals) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SIPG workload)",
            "config": {"workload": WORKLOAD, "dofs": pr.ndof, "rtol": RTOL, "lmax": LMAX},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "host_cores": os.cpu_count(), "sample": txt},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


MRHS_WORKLOAD = "sipg3d_p2_32cube_rhs32"
MRHS_LMAX = 100
# the 32-right-hand-side configuration at full size (64^3 p = 2 x 32 columns), timed over a
# bounded number of level-0 cycles beside single-column solves over the same cycles
C4_WORKLOAD = "sipg3d_p2_64cube_rhs32"
C4_CYCLES = 20
# the adjoint-gradient workload (log-normal coefficient, target field from the next seed)
ADJ_WORKLOAD = "sipg3d_p2_32cube_lognormal"
MRHS_PRECISION = "mixed_bf16"


# the batched FP32 sweep kernels the autotuner chooses from (kcmg_mrhs_tuning out[8])
SWEEP_KERNELS = {0: "tensor-core TF32x3 smoother sweeps (FP32 accumulation)",
                 1: "tensor-core TF32x3 smoother sweeps, bulk-copy staged (FP32 accumulation)",
                 2: "FP32 CUDA-core smoother sweeps"}
SWEEP_KERNEL_NAMES = {0: "k_msweep_tc", 1: "k_msweep_tcb", 2: "k_msweep_simt"}


def run_adjoint(pkg, dev):
    """One gradient evaluation of L(b, log nu) = 0.5 ||u - u_t||^2 with u = A(nu)^{-1} b on
    the log-normal workload, through torch.autograd: the forward solve (host assembly of
    A(nu), a new context, the solve) and the backward pass (the adjoint solve A^T lambda =
    u - u_t and the per-cell gradient kernel).  Timed on the host clock around each pass with
    a device synchronize (the forward pass includes host work), after one untimed
    evaluation.  value = DOFs x evaluations / s."""
    import numpy as np
    import torch

    from paper_2512_08728_gb300.autograd import KCycleSolve, SolveOptions, SWIPOperator
    from workloads import workload
    w = workload(ADJ_WORKLOAD)
    pr, pt = w.make(0), w.make(1)
    op = SWIPOperator(pr, options=SolveOptions(rtol=RTOL))
    b = torch.from_numpy(pr.b).to(dev)
    ut = op.solve(pt.nu, b)
    times = []
    for _ in range(2):
        log_nu = torch.from_numpy(np.log(pr.nu)).to(dev).requires_grad_(True)
        bb = b.clone().requires_grad_(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u = KCycleSolve.apply(bb, log_nu, op)
        loss = 0.5 * torch.sum((u - ut) ** 2)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        times.append((t1 - t0, time.perf_counter() - t1))
    fwd, bwd = times[-1]
    return {"value": pr.ndof / (fwd + bwd), "unit": UNIT, "workload": ADJ_WORKLOAD,
            "what": "one dL/db and dL/dlog nu evaluation (forward solve + adjoint solve + gradient)",
            "forward_s": fwd, "backward_s": bwd, "per_field_setup": op.last_setup,
            "grad_norm": float(torch.linalg.vector_norm(log_nu.grad)),
            "timing": "host clock with a device synchronize around each pass; one untimed evaluation first"}


def run_mrhs(pkg, rank, dev, stream, hbm_peak, args, wl_name=None, maxiter=None):
    """The batched form: 32 right-hand sides solved together (one K-cycle per column,
    shared operator applications, FP32 sweeps).  value = DOFs x columns / s."""
    import torch

    from workloads import workload
    wname = wl_name or args.mrhs_workload or MRHS_WORKLOAD
    cap = maxiter if maxiter is not None else args.maxiter
    prec_m = args.mrhs_precision or MRHS_PRECISION
    lmax_m = args.mrhs_lmax if args.mrhs_lmax is not None else MRHS_LMAX
    pm = workload(wname).make(rank)
    B = torch.from_numpy(pm.b).to(dev)
    X = torch.zeros_like(B)
    sm = pkg.KCycleSolver(pm, precision=prec_m, lmax=lmax_m, stream=stream.cuda_stream,
                          async_smooth=HEADLINE_ASYNC_M)
    pkg.kcmg_solve(sm.ctx, B, X, RTOL, 0.0, 1)   # build the batched engine and autotune
    tune = sm.mrhs_tuning()
    X.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    inf = pkg.kcmg_solve(sm.ctx, B, X, RTOL, 0.0, cap)
    e1.record(stream)
    torch.cuda.synchronize()
    mms = e0.elapsed_time(e1)
    # the same operator solved one column at a time (columns 0 and 1, FP64 and the same
    # mixed form) for comparison
    single = {}
    for prec in (() if args.no_single else ("fp64", prec_m)):
        s1 = pkg.KCycleSolver(pm, precision=prec, use_graph=True, lmax=200, stream=stream.cuda_stream,
                              async_smooth=HEADLINE_ASYNC_M)
        ts = []
        for j in (0, 1):
            bj = B[:, j].contiguous()
            xj = torch.zeros_like(bj)
            pkg.kcmg_solve(s1.ctx, bj, xj, RTOL, 0.0, 2)
            xj.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            ij = pkg.kcmg_solve(s1.ctx, bj, xj, RTOL, 0.0, cap)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append((e0.elapsed_time(e1), ij["iters"]))
        s1.close()
        single[prec] = {"value": pm.ndof * len(ts) / (sum(t for t, _ in ts) * 1e-3), "unit": UNIT,
                        "cycles": [c for _, c in ts],
                        "dof_cycles_per_s": pm.ndof * sum(c for _, c in ts) / (sum(t for t, _ in ts) * 1e-3)}
    sm.close()
    R = int(pm.b.shape[1])
    C = pm.ndof // pm.np_
    np2, S = pm.np_ * pm.np_, 2 * pm.d + 1
    inv_b = 2 if prec_m == "mixed_bf16" else 4
    # algorithmic bytes of one FP32 sweep (sweeps 2..5): FP32 off-diagonal blocks, stored
    # inverses, r (FP32) and the old and new iterates (FP32), each once
    sweep_bytes = C * ((S - 1) * np2 * 4 + np2 * inv_b) + 3 * pm.ndof * R * 4
    sweep_gbs = sweep_bytes / (tune["sweep_ms"] * 1e-3) / 1e9 if tune["sweep_ms"] > 0 else 0.0
    # FP64 block SpMM: one FMA per block element and column
    spmm_tflops = 2.0 * S * np2 * C * R / (tune["spmm_ms"] * 1e-3) / 1e12 if tune["spmm_ms"] > 0 else 0.0
    return {
        "value": pm.ndof * R / (mms * 1e-3), "unit": UNIT, "workload": wname, "nrhs": R,
        # DOF-cycles per second (columns x DOFs x level-0 cycles / s): comparable with the
        # single-column solves when --maxiter bounds both
        "dof_cycles_per_s": pm.ndof * R * inf["iters"] / (mms * 1e-3),
        "ms_per_step": mms, "status": inf["status"], "rel_res": inf["rel_res"],
        "cycles": inf["iters"], "level_iters": inf["level_iters"][:pm.nlevels],
        "lmax": lmax_m, "precision": prec_m, "kernel_launches": inf["kernel_launches"],
        "level0_cycle": f"Alg. AsyncMG, m = {HEADLINE_ASYNC_M} (every column)",
        "single_column_solves": single,
        "dtype": (SWEEP_KERNELS.get(int(tune["sweep_kernel"]), "?")
                  + (", BF16 block inverses" if prec_m == "mixed_bf16" else "")
                  + "; f64 residual minimisation, transfers, coarsest solve")
                 if prec_m != "fp64" else "f64",
        "autotuner": tune,
        "sweep": {"kernel": SWEEP_KERNEL_NAMES.get(int(tune["sweep_kernel"]), "?"),
                  "bound": "hbm", "achieved": sweep_gbs, "peak": hbm_peak, "unit": "GB/s",
                  "frac": sweep_gbs / hbm_peak, "bytes_per_launch": sweep_bytes,
                  "ms_per_launch": tune["sweep_ms"]},
        "spmm_fp64": {"bound": "alu", "achieved": spmm_tflops, "peak": FP64_TFLOPS,
                      "unit": "TFLOP/s", "frac": spmm_tflops / FP64_TFLOPS,
                      "ms_per_launch": tune["spmm_ms"]},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--probe", choices=["rm", "smooth"], default=None,
                    help="profiling runs only: on 48^3 p=2 (1.1M DOFs, 4 levels), 'rm' applies Alg. 1 "
                         "to --probe-n random corrections on level 0 (the k-th RM orthogonalises "
                         "against k - 1 vectors); 'smooth' runs three level-0 smoother calls and "
                         "operator applications; then exits")
    ap.add_argument("--probe-n", type=int, default=100)
    ap.add_argument("--probe-precision", default="fp64")
    ap.add_argument("--no-stretched", action="store_true",
                    help="skip the stretched p = 3 workload (48^3, 1:10 in z) of the mixed-precision forms")
    ap.add_argument("--all-forms", action="store_true",
                    help="also time the mixed forms with the multiplicative cycle (about 30 s each)")
    ap.add_argument("--async-m", type=int, default=None,
                    help="level-0 cycle of the headline solve: smoother steps of Alg. AsyncMG "
                         "(default %d); 0 = the multiplicative cycle of Alg. 2" % HEADLINE_ASYNC_M)
    ap.add_argument("--mrhs-only", action="store_true",
                    help="run only the batched form (profiling runs): skips the single-RHS solves")
    ap.add_argument("--mrhs-workload", default=None,
                    help="batched workload name (default %s)" % "sipg3d_p2_32cube_rhs32")
    ap.add_argument("--mrhs-precision", default=None, help="batched form precision (default mixed_bf16)")
    ap.add_argument("--mrhs-lmax", type=int, default=None, help="batched level-0 basis length")
    ap.add_argument("--no-single", action="store_true",
                    help="batched form: skip the single-column comparison solves")
    ap.add_argument("--mrhs", action="store_true",
                    help="also solve a 32-right-hand-side batch (32^3 p=2, 32 columns of U[-1,1]) "
                         "in the batched mixed form, with single-column solves of the same "
                         "operator beside it, and report it under forms")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint-gradient form (%s)" % ADJ_WORKLOAD)
    ap.add_argument("--no-c4", action="store_true",
                    help="skip the bounded 64^3 x 32-right-hand-side batched form (%d cycles)" % C4_CYCLES)
    ap.add_argument("--maxiter", type=int, default=MAXITER,
                    help="cap on level-0 cycles (profiling runs only; the benchmark solves to 1e-10)")
    ap.add_argument("--workload", default=WORKLOAD, help="workload name (profiling runs only)")
    ap.add_argument("--eager", action="store_true",
                    help="host-driven loop control instead of the CUDA graph (same kernels; "
                         "profilers see kernels inside conditional graph nodes only this way)")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import numpy as np
    import torch

    import paper_2512_08728_gb300 as pkg
    from workloads import workload

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    pkg.build()
    hbm_peak, peak_kind = _peaks()

    stream = torch.cuda.current_stream()
    if args.probe:
        from workloads import make_problem
        pp = make_problem(3, 2, (48, 48, 48), 4, seed=0)
        sv = pkg.KCycleSolver(pp, precision=args.probe_precision,
                              lmax=max(args.probe_n, 1), stream=stream.cuda_stream)
        if args.probe == "rm":
            zs = np.random.default_rng(1).standard_normal((args.probe_n, pp.ndof))
            _, rr, ll = sv.rm_sequence(0, pp.b, np.zeros(pp.ndof), zs)
            print(json.dumps({"probe": "rm", "basis": ll, "rnorm": float(np.linalg.norm(rr))}))
        else:
            rv = torch.from_numpy(pp.b).to(dev)
            for _ in range(3):
                zz = sv.smooth(0, rv)
                yy = sv.apply(0, rv)
            torch.cuda.synchronize()
            print(json.dumps({"probe": "smooth", "z": float(torch.linalg.vector_norm(zz)),
                              "y": float(torch.linalg.vector_norm(yy))}))
        sv.close()
        return
    if args.adjoint_only:
        if rank == 0:
            print(json.dumps({"adjoint": run_adjoint(pkg, dev)}), flush=True)
        return
    if args.mrhs_only:
        out = run_mrhs(pkg, rank, dev, stream, hbm_peak, args)
        if rank == 0:
            print(json.dumps({"mrhs": out}), flush=True)
        return
    pr = workload(args.workload).make(rank)
    head_m = HEADLINE_ASYNC_M if args.async_m is None else args.async_m
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    s = pkg.KCycleSolver(pr, precision="fp64", use_graph=not args.eager, lmax=LMAX,
                         async_smooth=head_m, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    b = torch.from_numpy(pr.b).to(dev)
    x = torch.zeros_like(b)

    def solve(sv, bb, xx, maxiter=None):
        xx.zero_()
        return pkg.kcmg_solve(sv.ctx, bb, xx, RTOL, 0.0, args.maxiter if maxiter is None else maxiter)

    # the first solve captures the CUDA graph; it is timed as part of the setup
    t0 = time.perf_counter()
    solve(s, b, x, maxiter=1)
    torch.cuda.synchronize()
    capture_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        info = solve(s, b, x)
    s.kernel_report()   # reset the coarse-cycle counters
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = ClockSampler(dev)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        infos.append(solve(s, b, x))
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = _max_over_ranks(e0.elapsed_time(e1), ws, dev)
    if ws > 1:
        torch.distributed.barrier()
    value = ws * pr.ndof * args.steps / (ms * 1e-3)
    status = [i["status"] for i in infos]
    rel = max(i["rel_res"] for i in infos)
    cycles = infos[-1]["iters"]
    lvl = infos[-1]["level_iters"]
    launches = sum(i["kernel_launches"] for i in infos)
    rep = s.kernel_report(reps=10)

    # The persistent coarse cycle times itself (GPU global timer at entry and after its
    # last barrier, accumulated over every launch of the timed region) and counts the
    # algorithmic bytes of every phase it runs.  Its data stays in the 129 MB L2 and its
    # arithmetic is FP64 (one FMA per 8-byte operand), so its roofline is the FP64 FMA
    # rate expressed as operand bytes per second; the HBM fraction is given beside it.
    # The level-0 operator and sweep kernels are timed standalone with CUDA events on the
    # library's stream (kernels inside a CUDA graph cannot be bracketed by events).
    fp64_gbs = FP64_TFLOPS * 1e3 / 2 * 8
    cl = max(1, rep["coarse_launches"])
    coarse_ms = rep["coarse_ms"] / cl
    coarse_bytes = rep["coarse_bytes"] / cl
    coarse_gbs = coarse_bytes / (coarse_ms * 1e-3) / 1e9 if coarse_ms > 0 else 0.0
    step_ms = ms / args.steps
    # Launches per solve of the level-0 and level-1 kernels, from the solve's own counts:
    # full sweeps (sweeps 2..5 of every smoother call; Alg. AsyncMG runs m smoother calls
    # per level-0 cycle, Alg. 2 two) and operator applications (one per RM: m + 1 per
    # level-0 cycle in Alg. AsyncMG, 3 in Alg. 2 and on level 1).  Their time per solve
    # is launches x the standalone CUDA-event time per launch.
    nsw = 4
    calls0 = head_m if head_m > 0 else 2
    rms0 = head_m + 1 if head_m > 0 else 3
    n_sweep = (cycles * calls0 * nsw, int(lvl[1]) * 2 * nsw)
    n_spmv = (cycles * rms0, int(lvl[1]) * 3)
    np_, S = pr.np_, 2 * pr.d + 1
    N0, N1 = pr.ndof, pr.ndof // (2 ** pr.d)
    sweep_flop = (2 * ((S - 1) * np_ + np_) * N0, 2 * ((S - 1) * np_ + np_) * N1)
    spmv_flop = (2 * S * np_ * N0, 2 * S * np_ * N1)

    def alu_kernel(name, what, t, n, flop):
        tot_ms = n[0] * t[0] + n[1] * t[1]
        tot_flop = n[0] * flop[0] + n[1] * flop[1]
        tf = tot_flop / (tot_ms * 1e-3) / 1e12 if tot_ms > 0 else 0.0
        return {"name": name, "what": what, "bound": "alu", "achieved": tf, "peak": FP64_TFLOPS,
                "unit": "TFLOP/s", "frac": tf / FP64_TFLOPS,
                "launches_per_step": {"level0": n[0], "level1": n[1]},
                "ms_per_launch": {"level0": t[0], "level1": t[1]},
                "flop_per_launch": {"level0": flop[0], "level1": flop[1]},
                "share_of_step": tot_ms / step_ms if step_ms > 0 else None,
                "timing": "standalone CUDA events per launch on the library's stream x launches "
                          "per solve (kernels inside the CUDA graph cannot be bracketed)"}

    kernels = [
        {"name": "k_coarse_cycle", "what": "persistent coarse cycle (levels below the first "
         "level with <= 100,000 rows)", "bound": "alu",
         "achieved": coarse_gbs, "peak": fp64_gbs, "unit": "GB/s",
         "frac": coarse_gbs / fp64_gbs, "hbm_frac": coarse_gbs / hbm_peak,
         "ms_per_launch": coarse_ms, "launches_per_step": rep["coarse_launches"] / args.steps,
         "bytes_per_launch": coarse_bytes, "share_of_step": rep["coarse_ms"] / ms if ms > 0 else 0.0,
         "timing": "GPU global timer inside the kernel over every launch of the timed region",
         "ms_per_launch_by_level": [v / cl for v in rep["coarse_level_ms"][:pr.nlevels]],
         "ms_per_launch_by_phase": {k: v / cl for k, v in rep["coarse_phase_ms"].items()}},
        alu_kernel("k_bj_sweep", "FP64 block-Jacobi sweep (Alg. BJ), levels 0 and 1",
                   (rep["sweep_ms"], rep["sweep1_ms"]), n_sweep, sweep_flop),
        alu_kernel("k_spmv", "FP64 operator application (Alg. 1: w = A z), levels 0 and 1",
                   (rep["spmv_ms"], rep["spmv1_ms"]), n_spmv, spmv_flop),
    ]
    # Alg. 1's Gram kernels on level 0 (one launch of each per level-0 RM), timed at the
    # basis length halfway through a restart period; level-1 launches are not counted
    n_rm0 = cycles * rms0
    for kname, key, what in (("k_gram_update", "gram_update", "Alg. 1 new column: w - W h, z - Z h (FP64), level 0"),
                             ("k_gram_dots", "gram_dots", "Alg. 1 first Gram pass: W^T w, ||w||^2 (FP64), level 0")):
        t, fl = rep[key + "_ms"], rep[key + "_flop"]
        tf = fl / (t * 1e-3) / 1e12 if t > 0 else 0.0
        kernels.append({"name": kname, "what": what, "bound": "alu", "achieved": tf, "peak": FP64_TFLOPS,
                        "unit": "TFLOP/s", "frac": tf / FP64_TFLOPS, "launches_per_step": n_rm0,
                        "ms_per_launch": t, "flop_per_launch": fl, "basis_length": rep["gram_l"],
                        "share_of_step": n_rm0 * t / step_ms if step_ms > 0 else None,
                        "timing": "standalone CUDA events per launch at the mid-restart basis length "
                                  "x level-0 RMs per solve"})
    # the dominant kernel: the largest share of the solve among the kernels timed here
    dom = max(kernels, key=lambda k: k["share_of_step"] or 0.0)
    traffic, traffic_note = _traffic(dom["name"])
    if traffic is not None and dom["name"] == "k_gram_update":   # bytes per unit -> per launch
        traffic = traffic * (2 * rep["gram_l"] + 5) * pr.ndof

    # end to end through the C interface with pinned host buffers: every step copies b
    # and x0 to the device and x back inside the timed region
    e2e = None
    if not args.no_e2e:
        k_e2e = max(1, min(args.steps, 3))
        bh = torch.from_numpy(pr.b).pin_memory().numpy()
        xh = torch.zeros(pr.ndof, dtype=torch.float64).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            xh[:] = 0.0
            pkg.kcmg_solve(s.ctx, bh, xh, RTOL, 0.0, args.maxiter)
        t_e2e = _max_over_ranks(time.perf_counter() - t0, ws, dev)
        e2e = {"value": ws * pr.ndof * k_e2e / t_e2e, "unit": UNIT, "steps": k_e2e,
               "h2d_bytes_per_step": 2 * pr.ndof * 8, "d2h_bytes_per_step": pr.ndof * 8,
               "host_buffers": "pinned"}
    s.close()

    # the other forms: one timed solve each, after the solve that captures its graph
    def time_form(prob, bb, xx, prec, am, smoother, lmax=LMAX, maxiter=None, matrix_free=False):
        skw = dict(smoother="as", omega=AS_OMEGA, sweeps=AS_SWEEPS) if smoother == "as" else {}
        if matrix_free:
            skw["matrix_free"] = True
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sm = pkg.KCycleSolver(prob, precision=prec, use_graph=True, lmax=lmax,
                              stream=stream.cuda_stream, async_smooth=am, **skw)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        solve(sm, bb, xx, maxiter=1)   # capture the graph
        sm.kernel_report()
        torch.cuda.synchronize()
        e0.record(stream)
        inf = solve(sm, bb, xx, maxiter=maxiter)
        e1.record(stream)
        torch.cuda.synchronize()
        mms = e0.elapsed_time(e1)
        rp = sm.kernel_report(reps=10)
        sm.close()
        ir = prec.startswith("ir32")
        if ir:
            dtype = ("f64 iterative refinement (compensated f64 residual) around an f32 inner "
                     "K-cycle: f32 operators, sweeps, transfers, bases"
                     + (", bf16 block inverses" if prec == "ir32_bf16" else "")
                     + "; f64 Gram reductions and coarsest solve")
        elif prec != "fp64":
            dtype = ("f32 smoother sweeps" + (", bf16 block inverses" if prec == "mixed_bf16" else "")
                     + "; f64 residual minimisation, transfers, coarsest solve")
        else:
            dtype = "f64"
        sw_peak = hbm_peak if prec != "fp64" else fp64_gbs
        return {
            "value": prob.ndof / (mms * 1e-3), "unit": UNIT, "timed_solves": 1,
            "ms_per_step": mms, "setup_s": setup, "status": inf["status"],
            "rel_res": inf["rel_res"], "cycles": inf["iters"],
            "refinements": inf["refinements"] if ir else None, "dtype": dtype,
            "cycle": ("Alg. 2 (multiplicative K-cycle)" if am == 0 else
                      f"Alg. AsyncMG on level 0: coarse path on a second stream, {am} smoother "
                      f"+ RM steps per cycle beside it"), "lmax": lmax,
            "smoother": ("Alg. AS: additive Schwarz on two partitions of overlapping 2^d-cell "
                         f"patches, omega {AS_OMEGA}, {AS_SWEEPS} sweeps" if smoother == "as"
                         else "Alg. BJ: block Jacobi, omega 0.7, 5 sweeps")
                        + ("; level-0 coupling matrix-free from the coefficient field and the face "
                           "reference matrices" if matrix_free else ""),
            "smoother_sweep": {"bound": "hbm" if prec != "fp64" else "alu",
                               "achieved": rp["sweep_bytes"] / (rp["sweep_ms"] * 1e-3) / 1e9,
                               "peak": sw_peak, "unit": "GB/s",
                               "frac": rp["sweep_bytes"] / (rp["sweep_ms"] * 1e-3) / 1e9 / sw_peak,
                               "ms_per_launch": rp["sweep_ms"]},
            "coarse_cycle_gbs": (rp["coarse_bytes"] / max(1, rp["coarse_launches"]))
                                / (rp["coarse_ms"] / max(1, rp["coarse_launches"]) * 1e-3) / 1e9
                                if rp["coarse_ms"] > 0 else None}

    forms = {}
    if not args.no_mixed:
        # (precision, level-0 cycle m, smoother) on the benchmark workload; each form runs
        # the level-0 cycle measured best for it over three seeds
        plan = [("fp64", 0, "bj"), ("mixed", HEADLINE_ASYNC_M, "bj"),
                ("mixed_bf16", HEADLINE_ASYNC_M, "bj"), ("fp64", AS_ASYNC_M_FP64, "as"),
                ("mixed_bf16", AS_ASYNC_M_MIXED, "as"),
                ("ir32", HEADLINE_ASYNC_M, "bj"), ("ir32_bf16", HEADLINE_ASYNC_M, "bj")]
        if args.all_forms:
            plan += [("mixed", 0, "bj"), ("mixed_bf16", 0, "bj")]
        for prec, am, smoother in plan:
            if prec == "fp64" and am == head_m and smoother == "bj":
                continue
            fname = (f"{prec}_multiplicative" if am == 0 else f"{prec}_task_parallel_m{am}")
            if smoother == "as":
                fname += "_schwarz"
            forms[fname] = time_form(pr, b, x, prec, am, smoother)
        # the FP32 sweeps with the level-0 coupling applied matrix-free from the coefficient field
        forms[f"mixed_bf16_task_parallel_m{HEADLINE_ASYNC_M}_matrix_free"] = time_form(
            pr, b, x, "mixed_bf16", HEADLINE_ASYNC_M, "bj", matrix_free=True)
        if not args.no_stretched and ws == 1:
            # the mixed-precision configuration: 48^3 cells, p = 3, stretched 1:10 in z, nu
            # 1:1e4 (block Jacobi stalls near 2e-4 on it; the Schwarz smoother converges)
            p3 = workload(STRETCHED).make(rank)
            b3 = torch.from_numpy(p3.b).to(dev)
            x3 = torch.zeros_like(b3)
            for prec in ("mixed", "fp64"):
                f = time_form(p3, b3, x3, prec, STRETCHED_ASYNC_M, "as")
                f["workload"] = STRETCHED
                forms[f"{STRETCHED}_{prec}_task_parallel_m{STRETCHED_ASYNC_M}_schwarz"] = f
            del b3, x3

    if args.mrhs:
        forms["mrhs32"] = run_mrhs(pkg, rank, dev, stream, hbm_peak, args)
    if not args.no_c4 and not args.no_mixed and ws == 1:
        # 64^3 x 32 right-hand sides, C4_CYCLES level-0 cycles: DOF-cycles per second beside
        # single-column solves of the same operator over the same number of cycles
        # (its bases take about 150 GB: a device without the room reports the failure here
        # and keeps the rest of the line)
        try:
            f = run_mrhs(pkg, rank, dev, stream, hbm_peak, args, wl_name=C4_WORKLOAD, maxiter=C4_CYCLES)
            f["bounded_cycles"] = C4_CYCLES
        except (pkg.KcmgError, RuntimeError) as e:   # the library's error, or torch's OOM
            f = {"error": str(e)}
        forms[f"{C4_WORKLOAD}_{C4_CYCLES}_cycles"] = f
    if not args.no_mixed and ws == 1:
        try:
            forms[f"{ADJ_WORKLOAD}_adjoint_gradient"] = run_adjoint(pkg, dev)
        except Exception as e:   # noqa: BLE001  (a failed form is reported; the line stands)
            forms[f"{ADJ_WORKLOAD}_adjoint_gradient"] = {"error": f"{type(e).__name__}: {e}"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v1, t1, txt1, _ = oracle_sample(pr, int(lvl[1]), int(cycles), async_m=head_m)
        cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
               "host_cores": os.cpu_count(), "sample": txt1}
        try:
            vn, tn, txtn, cores = oracle_sample(pr, int(lvl[1]), int(cycles), async_m=head_m,
                                                openmp=True)
            cpu = {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "host_cores": os.cpu_count(), "sample": txtn,
                   "single_core": {"value": v1, "unit": UNIT, "cores": 1, "sample": txt1}}
        except Exception as e:   # noqa: BLE001  (no OpenMP build on this host)
            cpu["all_core"] = f"unavailable: {e}"

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SIPG workload)",
            "config": {"workload": args.workload, "cells": list(pr.n), "p": pr.p, "dofs": pr.ndof,
                       "levels": pr.nlevels, "nu_ratio": 1000, "smoother": "block-Jacobi omega 0.7, 5 sweeps",
                       "rtol": RTOL, "lmax": LMAX, "cuda_graph": not args.eager, "coarse_cycle": "persistent",
                       "level0_cycle": (f"Alg. AsyncMG: coarse path on a second stream, {head_m} "
                                        "smoother + RM steps per cycle beside it (task-parallel OrthoMG)")
                                       if head_m > 0 else "Alg. 2 (multiplicative K-cycle)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "l2": "inputs larger than L2 (operator 1.47 GB vs 129 MB L2): no flush"},
            "setup_s": setup_s, "graph_capture_s": capture_s,
            "status": status, "rel_res": rel, "cycles": cycles, "level_iters": lvl[:pr.nlevels],
            "roofline": {"bound": dom["bound"], "achieved": dom["achieved"],
                         "peak": dom["peak"], "unit": dom["unit"], "frac": dom["frac"],
                         "traffic": traffic, "traffic_note": traffic_note,
                         "peak_kind": FP64_PEAK_NOTE + f"; HBM peak {hbm_peak} GB/s ({peak_kind})",
                         "kernel": dom["name"]},
            "kernels": kernels,
            "forms": forms,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
