"""Host-side checks of the C interface (no GPU needed): the library builds for sm_103a,
loads, and exports every entry point that include/kcmg.h declares; the binding fails
loudly when the library is missing."""
import os
import re

import pytest

import paper_2512_08728_gb300 as pkg
from paper_2512_08728_gb300 import kcmg as K

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kcmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kcmg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("kcmg_setup", "kcmg_solve", "kcmg_solve_adjoint", "kcmg_destroy"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = pkg.build()
    assert os.path.exists(path)
    lib = pkg.load_library()
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(K.exported_symbols()) == _declared()


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(K, "_lib", None)
    monkeypatch.setattr(K, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not found"):
        K.load_library()


def test_status_strings():
    lib = pkg.load_library()
    assert lib.kcmg_status_string(0) == b"ok"
    assert lib.kcmg_status_string(4).startswith(b"singular")


def test_default_params_follow_the_level_criteria():
    """kcmg_default_params (host only): the level criteria of Sec. 4.2 and Alg. BJ's
    omega and sweep count, the multiplicative cycle and three-product tensor-core sweeps."""
    p = K.kcmg_default_params(3, 10, (64, 64, 64), 5)
    assert (p.lvl_rtol[1], p.lvl_maxit[1]) == (0.1, 20)
    assert (p.lvl_rtol[2], p.lvl_maxit[2]) == (0.5, 2)
    assert all(p.lvl_maxit[l] == 1 for l in range(3, 5))
    assert abs(p.omega - 0.7) < 1e-15 and p.sweeps == 5
    assert p.async_smooth == 0 and p.tc_tf32_only == 0 and p.precision == K.KCMG_FP64


def test_solve_rejects_mismatched_shapes_before_any_device_call():
    import numpy as np
    pkg.load_library()
    with pytest.raises(ValueError):
        K.kcmg_solve(None, np.zeros(8), np.zeros(9))
    with pytest.raises(ValueError):
        K.kcmg_solve(None, np.zeros((8, 2, 2)), np.zeros((8, 2, 2)))
