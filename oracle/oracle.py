"""ctypes shim around kcmg_oracle.c (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

ORC_OK, ORC_NOT_CONVERGED, ORC_BREAKDOWN, ORC_NONFINITE, ORC_SINGULAR, ORC_INVALID_ARG = range(6)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kcmg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain -O2, single thread) or,
    with openmp=True, the same source with -fopenmp into liboracle_omp.so: its cell- and
    element-parallel loops then run on all host cores with bitwise the serial results."""
    lib = _LIB_OMP if openmp else _LIB
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".{os.getpid()}.tmp"
        flags = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *flags, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


def threads(n: int = 0) -> int:
    """Threads of the OpenMP build (n <= 0: all host cores); returns the count in use."""
    return int(_load(True).orc_threads(int(n)))


def _load(openmp: bool = False):
    with _lock:
        if openmp not in _libs:
            lib = C.CDLL(build(openmp=openmp))
            lib.orc_create.restype = C.c_void_p
            lib.orc_create.argtypes = [C.c_int, C.c_int, _ip, C.c_int, _dp, _dp, C.c_double,
                                       C.c_int, _dp, _ip, C.c_int, C.c_int, C.POINTER(C.c_int)]
            lib.orc_destroy.argtypes = [C.c_void_p]
            lib.orc_solve.restype = C.c_int
            lib.orc_solve.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_double, C.c_int,
                                      _dp, _ip, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_double), _ip]
            lib.orc_ncell.restype = C.c_int
            lib.orc_ncell.argtypes = [C.c_void_p, C.c_int]
            for nm in ("orc_apply", "orc_smooth", "orc_restrict", "orc_prolong"):
                getattr(lib, nm).argtypes = [C.c_void_p, C.c_int, _dp, _dp]
            lib.orc_coarse_solve.argtypes = [C.c_void_p, _dp, _dp]
            lib.orc_get_blocks.argtypes = [C.c_void_p, C.c_int, _dp]
            lib.orc_get_inv.argtypes = [C.c_void_p, C.c_int, _dp]
            lib.orc_rm_begin.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
            lib.orc_rm_call.restype = C.c_int
            lib.orc_rm_call.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, C.POINTER(C.c_int)]
            lib.orc_rm_basis.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
            lib.orc_restarts.restype = C.c_int
            lib.orc_restarts.argtypes = [C.c_void_p]
            lib.orc_set_async.argtypes = [C.c_void_p, C.c_int]
            lib.orc_basis_size.restype = C.c_int
            lib.orc_basis_size.argtypes = [C.c_void_p, C.c_int]
            lib.orc_grad_lognu.argtypes = [C.c_int, C.c_int, _ip, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            lib.orc_threads.restype = C.c_int
            lib.orc_threads.argtypes = [C.c_int]
            lib.orc_set_smoother.restype = C.c_int
            lib.orc_set_smoother.argtypes = [C.c_void_p, C.c_int]
            _libs[openmp] = lib
    return _libs[openmp]


def default_level_criteria(nlevels: int):
    """Sec. 4.2: level 1 stops at 0.1 r0 or 20 iterations, level 2 at 0.5 r0 or 2
    iterations, deeper levels run one iteration; level 0 is set per solve."""
    rtol = np.zeros(nlevels)
    maxit = np.ones(nlevels, dtype=np.int32)
    if nlevels > 1:
        rtol[1], maxit[1] = 0.1, 20
    if nlevels > 2:
        rtol[2], maxit[2] = 0.5, 2
    return rtol, maxit


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleSolver:
    """FP64 CPU K-cycle OrthoMG on a Cartesian block-ELL operator and its hierarchy."""

    def __init__(self, dim, np_, n, nlevels, blocks, prolong, omega=0.7, sweeps=5,
                 lvl_rtol=None, lvl_maxit=None, lmax=0, transpose=False, async_smooth=0,
                 openmp=False, smoother="bj"):
        self._lib = _load(openmp)
        rt, mi = default_level_criteria(nlevels)
        if lvl_rtol is not None:
            rt = np.asarray(lvl_rtol, dtype=np.float64)
        if lvl_maxit is not None:
            mi = np.asarray(lvl_maxit, dtype=np.int32)
        self.dim, self.np_, self.nlevels = dim, np_, nlevels
        self.n = np.array(list(n) + [1] * (3 - len(n)), dtype=np.int32)
        st = C.c_int(0)
        self._h = self._lib.orc_create(dim, np_, self.n, nlevels, _f64(blocks), _f64(prolong),
                                       float(omega), int(sweeps), _f64(rt),
                                       np.ascontiguousarray(mi, dtype=np.int32), int(lmax),
                                       int(transpose),
                                       C.byref(st))
        self.status = st.value
        if not self._h:
            raise RuntimeError(f"oracle setup failed with status {st.value}")
        # level 0 as Alg. AsyncMG with async_smooth smoother steps per cycle (0: Alg. 2)
        self._lib.orc_set_async(self._h, int(async_smooth))
        # smoother of every iterated level: "bj" (Alg. BJ) or "as" (Alg. AS, cell patches)
        if smoother not in ("bj", "as"):
            raise ValueError("smoother must be 'bj' or 'as'")
        if self._lib.orc_set_smoother(self._h, 1 if smoother == "as" else 0):
            raise RuntimeError("oracle: a Schwarz patch matrix is singular or too large")

    @classmethod
    def from_problem(cls, pr, **kw):
        return cls(pr.d, pr.np_, pr.n, pr.nlevels, pr.blocks, pr.prolong, **kw)

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    def ndof(self, level=0):
        return self._lib.orc_ncell(self._h, level) * self.np_

    def solve(self, b, x0=None, rtol=1e-10, atol=0.0, maxiter=500, hist_cap=4096):
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        hist = np.zeros(hist_cap)
        htype = np.zeros(hist_cap, dtype=np.int32)
        hl, it, rr = C.c_int(0), C.c_int(0), C.c_double(0)
        lit = np.zeros(16, dtype=np.int32)
        status = self._lib.orc_solve(self._h, b, x, rtol, atol, maxiter, hist, htype, hist_cap,
                                     C.byref(hl), C.byref(it), C.byref(rr), lit)
        info = {"status": status, "iters": it.value, "rel_res": rr.value,
                "hist": hist[:hl.value].copy(), "hist_type": htype[:hl.value].copy(),
                "level_iters": lit[:self.nlevels].copy(),
                "restarts": self._lib.orc_restarts(self._h)}
        return x, info

    def _vec(self, nm, level, x, nout):
        y = np.zeros(nout)
        getattr(self._lib, nm)(self._h, level, _f64(x), y)
        return y

    def apply(self, level, x):
        return self._vec("orc_apply", level, x, self.ndof(level))

    def smooth(self, level, b):
        return self._vec("orc_smooth", level, b, self.ndof(level))

    def restrict(self, level, r):
        return self._vec("orc_restrict", level, r, self.ndof(level + 1))

    def prolong(self, level, zc):
        return self._vec("orc_prolong", level, zc, self.ndof(level))

    def coarse_solve(self, r):
        z = np.zeros(self.ndof(self.nlevels - 1))
        self._lib.orc_coarse_solve(self._h, _f64(r), z)
        return z

    def blocks(self, level):
        out = np.zeros((2 * self.dim + 1, self.ndof(level) // self.np_, self.np_, self.np_))
        self._lib.orc_get_blocks(self._h, level, out)
        return out

    def inverses(self, level):
        out = np.zeros((self.ndof(level) // self.np_, self.np_, self.np_))
        self._lib.orc_get_inv(self._h, level, out)
        return out

    def rm_begin(self, level, b, x0):
        self._lib.orc_rm_begin(self._h, level, _f64(b), _f64(x0))

    def rm_call(self, level, z):
        N = self.ndof(level)
        x, r, l = np.zeros(N), np.zeros(N), C.c_int(0)
        rc = self._lib.orc_rm_call(self._h, level, _f64(z), x, r, C.byref(l))
        return rc, x, r, l.value

    def basis_size(self, level):
        return self._lib.orc_basis_size(self._h, level)

    def rm_basis(self, level, l):
        N = self.ndof(level)
        W, Z = np.zeros(l * N), np.zeros(l * N)
        self._lib.orc_rm_basis(self._h, level, W, Z)
        return W.reshape(l, N), Z.reshape(l, N)


def grad_lognu(pr, nu, lam, u):
    """g_K = -lambda^T (dA/d log nu_K) u for the SWIP operator of problem pr."""
    lib = _load()
    n = np.array(list(pr.n) + [1] * (3 - len(pr.n)), dtype=np.int32)
    g = np.zeros(int(np.prod(pr.n)))
    lib.orc_grad_lognu(pr.d, pr.np_, n, _f64(nu), _f64(pr.ref["V"]), _f64(pr.ref["F"]),
                       _f64(pr.ref["B"]), _f64(lam), _f64(u), g)
    return g
