"""Thin Python binding of libkcmg (include/kcmg.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may be NumPy
arrays (host memory: the library stages them, so copies are part of the call) or torch
tensors on the GPU (device memory: no staging).  All vectors are float64 and contiguous.
There is no fallback: if libkcmg.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

KCMG_MAX_LEVELS = 12
KCMG_OK, KCMG_NOT_CONVERGED, KCMG_BREAKDOWN, KCMG_NONFINITE, KCMG_SINGULAR, \
    KCMG_INVALID_ARG, KCMG_OOM, KCMG_CUDA_ERROR = range(8)
KCMG_FP64, KCMG_MIXED, KCMG_MIXED_BF16INV, KCMG_IR32, KCMG_IR32_BF16INV = range(5)
PRECISIONS = {"fp64": KCMG_FP64, "mixed": KCMG_MIXED, "mixed_bf16": KCMG_MIXED_BF16INV,
              "ir32": KCMG_IR32, "ir32_bf16": KCMG_IR32_BF16INV}
# phase kinds of the coarse-cycle kernel's timers (kcmg_kernel_report out[19 + k])
COARSE_PHASES = ["sweep", "rm_gram1", "rm_reorth", "rm_update", "rm_finish", "transfer",
                 "coarsest", "restart", "control"]


class kcmg_params(C.Structure):
    _fields_ = [("dim", C.c_int), ("np", C.c_int), ("n", C.c_int * 3), ("nlevels", C.c_int),
                ("blocks", C.c_void_p), ("prolong", C.c_void_p), ("omega", C.c_double),
                ("sweeps", C.c_int), ("lvl_rtol", C.c_double * KCMG_MAX_LEVELS),
                ("lvl_maxit", C.c_int * KCMG_MAX_LEVELS), ("lmax", C.c_int),
                ("precision", C.c_int), ("use_graph", C.c_int), ("coarse_persistent", C.c_int),
                ("tc_tf32_only", C.c_int), ("async_smooth", C.c_int),
                ("ir_inner_rtol", C.c_double), ("ir_max_steps", C.c_int),
                ("ir_inner_maxit", C.c_int), ("smoother", C.c_int),
                ("mf_nu", C.c_void_p), ("mf_F", C.c_void_p)]


class kcmg_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("level_iters", C.c_int * KCMG_MAX_LEVELS),
                ("restarts", C.c_int), ("refinements", C.c_int), ("res0", C.c_double),
                ("rel_res", C.c_double), ("kernel_launches", C.c_longlong),
                ("hist_cap", C.c_int), ("hist_len", C.c_int),
                ("hist", C.c_void_p), ("hist_type", C.c_void_p)]


class KcmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"kcmg status {status}: {msg}")
        self.status = status


_lib = None


def load_library():
    """Load libkcmg.so from the in-tree build directory (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"libkcmg.so not found at {LIB}: run paper_2512_08728_gb300.build()")
    lib = C.CDLL(LIB)
    vp, ip, dp = C.c_void_p, C.c_int, C.c_double
    sig = {
        "kcmg_default_params": (None, [C.POINTER(kcmg_params), ip, ip, C.POINTER(C.c_int), ip]),
        "kcmg_setup": (ip, [C.POINTER(vp), C.POINTER(kcmg_params), vp]),
        "kcmg_solve": (ip, [vp, vp, vp, ip, dp, dp, ip, C.POINTER(kcmg_info)]),
        "kcmg_solve_adjoint": (ip, [vp, vp, vp, ip, dp, dp, ip, C.POINTER(kcmg_info)]),
        "kcmg_grad_lognu": (ip, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "kcmg_apply": (ip, [vp, ip, ip, vp, vp]),
        "kcmg_smooth": (ip, [vp, ip, vp, vp]),
        "kcmg_restrict": (ip, [vp, ip, vp, vp]),
        "kcmg_prolong": (ip, [vp, ip, vp, vp]),
        "kcmg_coarse_solve": (ip, [vp, vp, vp]),
        "kcmg_get_blocks": (ip, [vp, ip, vp]),
        "kcmg_rm_sequence": (ip, [vp, ip, vp, vp, vp, ip, vp, vp, C.POINTER(C.c_int)]),
        "kcmg_level_cells": (ip, [vp, ip]),
        "kcmg_kernel_report": (ip, [vp, ip, vp, ip]),
        "kcmg_residual_noalloc": (ip, [vp, vp, vp, vp, C.POINTER(C.c_double)]),
        "kcmg_mrhs_tuning": (ip, [vp, vp, ip]),
        "kcmg_apply_multi": (ip, [vp, ip, ip, vp, vp]),
        "kcmg_smooth_multi": (ip, [vp, ip, ip, vp, vp]),
        "kcmg_last_error": (C.c_char_p, [vp]),
        "kcmg_status_string": (C.c_char_p, [ip]),
        "kcmg_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return ["kcmg_default_params", "kcmg_setup", "kcmg_solve", "kcmg_solve_adjoint",
            "kcmg_grad_lognu", "kcmg_apply", "kcmg_smooth", "kcmg_restrict", "kcmg_prolong",
            "kcmg_coarse_solve", "kcmg_get_blocks", "kcmg_rm_sequence", "kcmg_level_cells",
            "kcmg_kernel_report", "kcmg_residual_noalloc", "kcmg_mrhs_tuning",
            "kcmg_apply_multi", "kcmg_smooth_multi",
            "kcmg_last_error", "kcmg_status_string", "kcmg_destroy"]


# ---------------------------------------------------------------- marshalling helpers
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, write=False):
    """(pointer, keepalive) of a float64 contiguous host array or torch tensor."""
    if a is None:
        return None, None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise ValueError("expected a contiguous numpy array or torch tensor")
    if write and not a.flags.writeable:
        raise ValueError("output array is read-only")
    return a.ctypes.data, a


def _f64(a):
    if _is_torch(a):
        import torch
        return a.to(torch.float64).contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _empty_like(a, n):
    if _is_torch(a):
        import torch
        return torch.empty(n, dtype=torch.float64, device=a.device)
    return np.empty(n, dtype=np.float64)


def _check(ctx, st):
    if st not in (KCMG_OK, KCMG_NOT_CONVERGED):
        lib = load_library()
        raise KcmgError(st, lib.kcmg_last_error(ctx).decode())
    return st


# ---------------------------------------------------------------- C entry points
def kcmg_default_params(dim, np_, n, nlevels):
    p = kcmg_params()
    nn = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    load_library().kcmg_default_params(C.byref(p), dim, np_, nn, nlevels)
    return p


def kcmg_setup(params: kcmg_params, blocks, prolong, stream=None):
    """Returns the context handle (int).  blocks/prolong: float64 host or device arrays."""
    lib = load_library()
    blocks, prolong = _f64(blocks), _f64(prolong)
    params.blocks, _ = _ptr(blocks)
    params.prolong, _ = _ptr(prolong)
    h = C.c_void_p()
    st = lib.kcmg_setup(C.byref(h), C.byref(params), stream)
    if st != KCMG_OK:
        msg = lib.kcmg_last_error(h).decode() if h.value else "setup failed"
        if h.value:
            lib.kcmg_destroy(h)
        raise KcmgError(st, msg)
    return h.value


def kcmg_destroy(ctx):
    if ctx:
        load_library().kcmg_destroy(ctx)


def _info(hist_cap):
    info = kcmg_info()
    hist = np.zeros(max(hist_cap, 1))
    htype = np.zeros(max(hist_cap, 1), dtype=np.int32)
    info.hist_cap = hist_cap
    info.hist = hist.ctypes.data if hist_cap else None
    info.hist_type = htype.ctypes.data if hist_cap else None
    return info, hist, htype


def _info_dict(st, info, hist, htype):
    n = info.hist_len
    return {"status": st, "iters": info.iters, "level_iters": list(info.level_iters),
            "restarts": info.restarts, "refinements": info.refinements, "res0": info.res0,
            "rel_res": info.rel_res, "kernel_launches": info.kernel_launches,
            "hist": hist[:n].copy(), "hist_type": htype[:n].copy()}


def kcmg_solve(ctx, b, x, rtol=1e-10, atol=0.0, maxiter=500, hist_cap=4096, adjoint=False):
    """Solve in place: x holds x0 on entry and the solution on return.  b, x: [N] or
    [N, nrhs] (nrhs <= 32, right-hand sides fastest)."""
    lib = load_library()
    if tuple(b.shape) != tuple(x.shape) or len(b.shape) not in (1, 2):
        raise ValueError("b and x must have the same shape [N] or [N, nrhs]")
    nrhs = 1 if len(b.shape) == 1 else int(b.shape[1])
    pb, kb = _ptr(b)
    px, kx = _ptr(x, write=True)
    info, hist, htype = _info(hist_cap)
    f = lib.kcmg_solve_adjoint if adjoint else lib.kcmg_solve
    st = f(ctx, pb, px, nrhs, float(rtol), float(atol), int(maxiter), C.byref(info))
    _check(ctx, st)
    return _info_dict(st, info, hist, htype)


def kcmg_solve_adjoint(ctx, g, lam, rtol=1e-10, atol=0.0, maxiter=500, hist_cap=4096):
    return kcmg_solve(ctx, g, lam, rtol, atol, maxiter, hist_cap, adjoint=True)


def _multi(name, ctx, level, a):
    if len(a.shape) != 2:
        raise ValueError("expected an [N, nrhs] array")
    out = _empty_like(a, tuple(a.shape))
    pa, ka = _ptr(_f64(a))
    po, ko = _ptr(out, write=True)
    _check(ctx, getattr(load_library(), name)(ctx, level, int(a.shape[1]), pa, po))
    return out


def kcmg_apply_multi(ctx, level, x):
    """Y = A_level X for X [N_level, nrhs] (FP64 batched operator kernel)."""
    return _multi("kcmg_apply_multi", ctx, level, x)


def kcmg_smooth_multi(ctx, level, r):
    """Z = BJ_level(R) for R [N_level, nrhs] (batched sweeps in the context's precision)."""
    return _multi("kcmg_smooth_multi", ctx, level, r)


def kcmg_mrhs_tuning(ctx):
    """Launch shapes the multi-right-hand-side autotuner chose (see kcmg.h)."""
    out = np.zeros(9)
    _check(ctx, load_library().kcmg_mrhs_tuning(ctx, out.ctypes.data, out.size))
    keys = ["spmm_warps", "spmm_ms", "sweep_warps", "sweep_grid", "sweep_ms", "lcap0", "nrhs",
            "x3", "sweep_kernel"]
    return dict(zip(keys, out.tolist()))


def kcmg_level_cells(ctx, level):
    return load_library().kcmg_level_cells(ctx, level)


def kcmg_residual_noalloc(ctx, b, x, r):
    """r = b - A x (finest-level FP64 operator) without any device allocation; b, x, r are
    device tensors.  Returns ||r||.  See kcmg.h for the scratch it shares across calls."""
    for a in (b, x, r):
        if not (_is_torch(a) and a.is_cuda and a.dtype.is_floating_point and a.element_size() == 8):
            raise ValueError("kcmg_residual_noalloc takes float64 CUDA tensors")
    nrm = C.c_double(0.0)
    _check(ctx, load_library().kcmg_residual_noalloc(ctx, _ptr(b)[0], _ptr(x)[0],
                                                     _ptr(r, write=True)[0], C.byref(nrm)))
    return nrm.value


def kcmg_kernel_report(ctx, reps=0):
    """Coarse-cycle kernel counters since the last call and, with reps > 0, CUDA-event
    timings of the level-0 operator application and smoother sweep (see kcmg.h)."""
    n0 = 7 + KCMG_MAX_LEVELS + len(COARSE_PHASES)
    out = np.zeros(n0 + 9)
    _check(ctx, load_library().kcmg_kernel_report(ctx, int(reps), out.ctypes.data, out.size))
    ph = out[7 + KCMG_MAX_LEVELS:n0]
    return {"coarse_launches": int(out[0]), "coarse_ms": out[1], "coarse_bytes": out[2],
            "spmv_ms": out[3], "spmv_bytes": out[4], "sweep_ms": out[5], "sweep_bytes": out[6],
            "coarse_level_ms": out[7:7 + KCMG_MAX_LEVELS].tolist(),
            "coarse_phase_ms": dict(zip(COARSE_PHASES, ph.tolist())),
            "spmv1_ms": out[n0], "spmv1_bytes": out[n0 + 1], "sweep1_ms": out[n0 + 2],
            "sweep1_bytes": out[n0 + 3], "gram_dots_ms": out[n0 + 4], "gram_dots_flop": out[n0 + 5],
            "gram_update_ms": out[n0 + 6], "gram_update_flop": out[n0 + 7],
            "gram_l": int(out[n0 + 8])}


def _unary(name, ctx, level, x, nout, *extra):
    lib = load_library()
    x = _f64(x)
    y = _empty_like(x, nout)
    px, _ = _ptr(x)
    py, _ = _ptr(y, write=True)
    args = [ctx] + ([level] if level is not None else []) + list(extra) + [px, py]
    _check(ctx, getattr(lib, name)(*args))
    return y


def kcmg_apply(ctx, level, x, op=0, np_=None):
    n = kcmg_level_cells(ctx, level) * np_
    return _unary("kcmg_apply", ctx, level, x, n, op)


def kcmg_smooth(ctx, level, r, np_):
    return _unary("kcmg_smooth", ctx, level, r, kcmg_level_cells(ctx, level) * np_)


def kcmg_restrict(ctx, level, r, np_):
    return _unary("kcmg_restrict", ctx, level, r, kcmg_level_cells(ctx, level + 1) * np_)


def kcmg_prolong(ctx, level, zc, np_):
    return _unary("kcmg_prolong", ctx, level, zc, kcmg_level_cells(ctx, level) * np_)


def kcmg_coarse_solve(ctx, r):
    return _unary("kcmg_coarse_solve", ctx, None, r, int(np.asarray(r).shape[0]) if not _is_torch(r) else r.numel())


def kcmg_get_blocks(ctx, level, dim, np_):
    lib = load_library()
    out = np.zeros((2 * dim + 1, kcmg_level_cells(ctx, level), np_, np_))
    _check(ctx, lib.kcmg_get_blocks(ctx, level, out.ctypes.data))
    return out


def kcmg_rm_sequence(ctx, level, b, x0, zs, np_):
    lib = load_library()
    N = kcmg_level_cells(ctx, level) * np_
    b, x0 = _f64(b), _f64(x0)
    zs = np.ascontiguousarray(zs, dtype=np.float64).reshape(-1, N) if len(zs) else np.zeros((0, N))
    x, r, l = np.zeros(N), np.zeros(N), C.c_int(0)
    _check(ctx, lib.kcmg_rm_sequence(ctx, level, _ptr(b)[0], _ptr(x0)[0],
                                     zs.ctypes.data if zs.size else None, zs.shape[0],
                                     x.ctypes.data, r.ctypes.data, C.byref(l)))
    return x, r, l.value


def kcmg_grad_lognu(ctx, nu, V, F, B, lam, u):
    lib = load_library()
    arrs = [_f64(a) for a in (nu, V, F, B, lam, u)]
    g = _empty_like(arrs[-1], int(arrs[0].shape[0]) if not _is_torch(arrs[0]) else arrs[0].numel())
    ptrs = [_ptr(a)[0] for a in arrs]
    _check(ctx, lib.kcmg_grad_lognu(ctx, *ptrs, _ptr(g, write=True)[0]))
    return g


# ---------------------------------------------------------------- convenience wrapper
class KCycleSolver:
    """Owns one kcmg context built from a workloads.Problem-like object."""

    def __init__(self, problem, precision="fp64", use_graph=True, omega=0.7, sweeps=5,
                 lmax=0, lvl_rtol=None, lvl_maxit=None, coarse_persistent=True, stream=None,
                 tc_tf32_only=0, async_smooth=0, ir_inner_rtol=None, ir_max_steps=None,
                 ir_inner_maxit=None, smoother="bj", matrix_free=False):
        pr = problem
        self.dim, self.np_, self.nlevels = pr.d, pr.np_, pr.nlevels
        self.ndof = pr.ndof
        p = kcmg_default_params(pr.d, pr.np_, pr.n, pr.nlevels)
        p.omega, p.sweeps, p.lmax = omega, sweeps, lmax
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.use_graph = int(use_graph)
        p.coarse_persistent = int(coarse_persistent)
        p.tc_tf32_only = int(tc_tf32_only)
        p.async_smooth = int(async_smooth)
        if ir_inner_rtol is not None:
            p.ir_inner_rtol = float(ir_inner_rtol)
        if ir_max_steps is not None:
            p.ir_max_steps = int(ir_max_steps)
        if ir_inner_maxit is not None:
            p.ir_inner_maxit = int(ir_inner_maxit)
        if smoother not in ("bj", "as"):
            raise ValueError("smoother must be 'bj' (Alg. BJ) or 'as' (Alg. AS)")
        p.smoother = 1 if smoother == "as" else 0
        keep = []
        if matrix_free:   # level-0 FP32 sweeps from the coefficient field and face matrices
            nu = np.ascontiguousarray(pr.nu, dtype=np.float64)
            Fm = np.ascontiguousarray(pr.ref["F"], dtype=np.float64)
            p.mf_nu, p.mf_F = nu.ctypes.data, Fm.ctypes.data
            keep = [nu, Fm]
        if lvl_rtol is not None:
            for i, v in enumerate(lvl_rtol):
                p.lvl_rtol[i] = v
        if lvl_maxit is not None:
            for i, v in enumerate(lvl_maxit):
                p.lvl_maxit[i] = v
        self.params = p
        self.ctx = kcmg_setup(p, pr.blocks, pr.prolong, stream)
        del keep

    def close(self):
        if getattr(self, "ctx", None):
            kcmg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def solve(self, b, x0=None, rtol=1e-10, atol=0.0, maxiter=500, adjoint=False):
        b = _f64(b)
        if x0 is None:
            x = _empty_like(b, tuple(b.shape))
            x[:] = 0
        else:
            x = _f64(x0).clone() if _is_torch(x0) else _f64(x0).copy()
        info = kcmg_solve(self.ctx, b, x, rtol, atol, maxiter, adjoint=adjoint)
        return x, info

    def apply(self, level, x, op=0):
        return kcmg_apply(self.ctx, level, x, op, self.np_)

    def smooth(self, level, r):
        return kcmg_smooth(self.ctx, level, r, self.np_)

    def restrict(self, level, r):
        return kcmg_restrict(self.ctx, level, r, self.np_)

    def prolong(self, level, zc):
        return kcmg_prolong(self.ctx, level, zc, self.np_)

    def coarse_solve(self, r):
        return kcmg_coarse_solve(self.ctx, r)

    def blocks(self, level):
        return kcmg_get_blocks(self.ctx, level, self.dim, self.np_)

    def rm_sequence(self, level, b, x0, zs):
        return kcmg_rm_sequence(self.ctx, level, b, x0, zs, self.np_)

    def apply_multi(self, level, x):
        return kcmg_apply_multi(self.ctx, level, x)

    def smooth_multi(self, level, r):
        return kcmg_smooth_multi(self.ctx, level, r)

    def mrhs_tuning(self):
        return kcmg_mrhs_tuning(self.ctx)

    def kernel_report(self, reps=0):
        return kcmg_kernel_report(self.ctx, reps)

    def grad_lognu(self, nu, ref, lam, u):
        return kcmg_grad_lognu(self.ctx, nu, ref["V"], ref["F"], ref["B"], lam, u)
