"""The binary128 divided-difference scheme (LL_DD_TABLE_Q) on the device path (needs a GB300).

The forward and the batched launch take their Newton coefficients from the chosen scheme; the
binary128 table and Algorithm 1 give the same coefficients to rounding, so the estimates agree
with each other and with the oracle at the parity bar.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from synth import laplacian_2d
from tests.gpu_util import TOL, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_forward_with_binary128_coefficients(L, h, prec):
    A = laplacian_2d(40, 0.01)   # condition number about 800
    lo, hi = 0.01, 8.01
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    auto = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=80, probes=30, seed=3, precision=prec))
    assert h.info()["taylor_terms"] > 0
    q = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=80, probes=30, seed=3, precision=prec, dd_scheme="table_q"))
    assert h.info()["taylor_terms"] == 0
    assert abs(q - auto) <= 1e-12 * abs(auto)
    want = O.logdet_leja(A, lo, hi, 80, 30, 3, f32=(prec == "f32"))["estimate"]
    assert abs(q - want) / abs(want) < TOL[prec]


def test_batched_with_binary128_coefficients(L, h):
    mats = [laplacian_2d(n, t) for n, t in ((30, 0.05), (45, 0.5), (23, 0.01))]
    dm = [L.DeviceCSR.from_host(A) for A in mats]
    bounds = [(t, 8.0 + t) for t in (0.05, 0.5, 0.01)]
    auto = np.array(L.ll_logdet_batched(h, dm, bounds, L.options(probes=24, seed=1)))
    q = np.array(L.ll_logdet_batched(h, dm, bounds, L.options(probes=24, seed=1, dd_scheme="table_q")))
    assert np.all(np.abs(q - auto) <= 1e-12 * np.abs(auto))


def test_unknown_scheme_is_an_error(L, h):
    A = laplacian_2d(10, 0.1)
    o = L.options(degree=10, probes=6)
    o.dd_scheme = 7
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_forward(h, L.DeviceCSR.from_host(A), 0.1, 8.1, o)
    assert ei.value.name == "LL_ERR_INVALID_ARG"
