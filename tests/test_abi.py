"""The C-ABI library builds, loads without a GPU, and exports every entry point include/leja.h
declares; host-side entry points agree bit for bit with the oracle (CPU only)."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions() -> list[str]:
    text = open(os.path.join(ROOT, "include", "leja.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ll_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2603_02207_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ["ll_create", "ll_destroy", "ll_leja_points", "ll_divided_differences", "ll_gershgorin",
                 "ll_probes", "ll_apply_poly", "ll_logdet_forward", "ll_logdet_backward", "ll_logdet_batched",
                 "ll_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2603_02207_gb300 import _ffi
    assert set(_declared_functions()) <= set(_ffi.SIGNATURES)


def test_host_leja_points_bit_exact_with_oracle(libpath):
    from oracle.leja import fast_leja_points
    import paper_2603_02207_gb300 as L
    assert np.array_equal(L.ll_leja_points(300), fast_leja_points(300))


@pytest.mark.parametrize("lmin,lmax,m", [(1.0, 81.0, 39), (1.0, 241.0, 120), (0.1, 8.1, 39), (1.0, 8080.0, 80),
                                          (1.0, 2.5e6, 150), (0.01, 3e4, 150)])
def test_host_divided_differences_match_oracle(libpath, lmin, lmax, m):
    from oracle import logdet as O
    import paper_2603_02207_gb300 as L
    d, terms = L.ll_divided_differences(lmin, lmax, m)
    _, _, _, do, po = O.newton_leja_setup(lmin, lmax, m)
    assert terms == po
    assert np.max(np.abs(d - do)) <= 1e-13 * np.max(np.abs(do))


def test_host_entry_points_reject_bad_arguments(libpath):
    from paper_2603_02207_gb300 import _ffi
    import paper_2603_02207_gb300 as L
    lib = _ffi.load()
    out = np.zeros(4)
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.ll_leja_points(-1, p) == 1
    assert lib.ll_divided_differences(_ffi.ll_bounds(0.0, 1.0), 3, 0, p, None) == 3
    assert lib.ll_divided_differences(_ffi.ll_bounds(2.0, 1.0), 3, 0, p, None) == 3
    assert lib.ll_divided_differences(_ffi.ll_bounds(1.0, 2.0), 3, 7, p, None) == 1
    assert lib.ll_status_string(5) == b"LL_ERR_QR_BREAKDOWN"
    # handle setters refuse a null handle before touching the device
    assert lib.ll_set_adjoint_fusion(None, _ffi.LL_FUSE_ON) == 1
    assert lib.ll_set_keep_budget(None, 0) == 1
    # a condition number of 1e7 switches to the divided-difference table (0 Taylor terms)
    d, terms = L.ll_divided_differences(1.0, 1e7, 60)
    assert terms == 0 and np.all(np.isfinite(d))


@pytest.mark.parametrize("lmin,lmax,m", [(1.0, 81.0, 39), (1.0, 8080.0, 80), (1.0, 2.5e6, 150), (1.0, 1e9, 250),
                                          (0.01, 3e4, 150), (1.0, 1e12, 250), (0.37, 2.9, 7)])
def test_host_binary128_table_is_the_rounded_exact_coefficients(libpath, lmin, lmax, m):
    """LL_DD_TABLE_Q: every d_j is within rounding of the 120-digit table at the library's own
    nodes c + gamma xi_i (c, gamma in FP64), at any conditioning; Algorithm 1's long series
    (kappa = 8080: 117,022 terms) is 3.5e-14 off, the FP64 table up to 4e-12."""
    from oracle.leja import fast_leja_points
    import paper_2603_02207_gb300 as L
    from tests import pins
    d = L.ll_divided_differences_q(lmin, lmax, m)
    ref = pins.hp_scaled_divided_differences(lmin, lmax, fast_leja_points(m + 1),
                                             c_g=((lmin + lmax) / 2.0, (lmax - lmin) / 4.0))
    assert np.max(np.abs(d - ref)) <= 2.5e-16 * np.max(np.abs(ref))


def test_host_binary128_table_rejects_bad_arguments(libpath):
    from paper_2603_02207_gb300 import _ffi
    lib = _ffi.load()
    out = np.zeros(4)
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.ll_divided_differences_q(_ffi.ll_bounds(0.0, 1.0), 3, p) == 3
    assert lib.ll_divided_differences_q(_ffi.ll_bounds(2.0, 1.0), 3, p) == 3
    assert lib.ll_divided_differences_q(_ffi.ll_bounds(1.0, 2.0), -1, p) == 1
    assert lib.ll_divided_differences_q(_ffi.ll_bounds(1.0, 2.0), 3, None) == 1


def _header_constants() -> dict[str, int]:
    """LL_ constants of include/leja.h: enumerators with explicit values and #define'd integers."""
    text = open(os.path.join(ROOT, "include", "leja.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for name, val in re.findall(r"\b(LL_[A-Z0-9_]+)\s*=\s*([0-9]+)\s*[,}]", text):
        out[name] = int(val)
    for name, expr in re.findall(r"#define\s+(LL_[A-Z0-9_]+)\s+\(?([0-9 <]+)\)?", text):
        out[name] = int(eval(expr, {"__builtins__": {}}))   # digits and shifts only
    return out


def test_binding_constants_equal_the_header():
    """Every LL_ integer the ctypes binding defines is declared in the header with that value."""
    from paper_2603_02207_gb300 import _ffi
    hdr = _header_constants()
    ours = {k: v for k, v in vars(_ffi).items() if k.startswith("LL_") and isinstance(v, int)}
    assert ours, "no constants in the binding"
    missing = sorted(k for k in ours if k not in hdr)
    assert not missing, missing
    wrong = sorted(k for k, v in ours.items() if hdr[k] != v)
    assert not wrong, {k: (ours[k], hdr[k]) for k in wrong}
