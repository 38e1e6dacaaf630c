"""The GMRF of the paper's maximum-likelihood experiment (Section 5.3) on the GPU: log det Q(theta)
and d/dtheta log det Q(theta), Q(theta) = I + theta Adj on a 4-neighbour grid, against the
oracle and the closed forms (needs a GB300 and the library)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from synth import CSR, gmrf_theta
from tests import pins
from tests.gpu_util import TOL, lib, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


def _dtheta_values(A) -> np.ndarray:
    """d a_e / d theta: 1 on the neighbour entries, 0 on the diagonal."""
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    return (np.asarray(A.colind) != rows).astype(np.float64)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("theta", [-0.22, 0.15])
def test_gmrf_theta_forward_matches_oracle(L, h, prec, theta):
    """48 x 48 grid, Gershgorin bounds [1 - 4|theta|, 1 + 4|theta|] (sigma = 1 - 4|theta|), degree
    from the bounds, 30 Rademacher probes."""
    A = gmrf_theta(48, theta)
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    lo, hi = L.ll_gershgorin(h, dA)
    stored = A if prec != "f32" else CSR(A.n, A.rowptr, A.colind, A.values.astype(np.float32).astype(np.float64))
    assert (lo, hi) == O.gershgorin(stored)
    m = O.degree_from_bounds(lo, hi)
    got = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=m, probes=30, seed=4, precision=prec))
    want = O.logdet_leja(A, lo, hi, m, 30, 4, f32=(prec == "f32"))["estimate"]
    assert abs(got - want) / abs(want) < TOL[prec]
    assert h.info()["sigma"] == pytest.approx(1 - 4 * abs(theta), abs=1e-15 if prec != "f32" else 1e-7)


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_gmrf_theta_gradient_matches_oracle(L, h, prec):
    """The frozen-basis gradient with respect to every stored value, and its chain to theta
    (d a_e / d theta = 1 on the neighbour entries), against the oracle's reverse recurrence."""
    torch = need_gpu()
    theta = -0.22
    A = gmrf_theta(30, theta)
    lo, hi = O.gershgorin(A)
    m = O.degree_from_bounds(lo, hi)
    dA = L.DeviceCSR.from_host(A)
    L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=m, probes=24, seed=7, precision=prec, keep_for_backward=True))
    g = L.ll_logdet_backward(h, dA, 1.0)
    ref = O.logdet_leja(A, lo, hi, m, 24, 7)
    want = O.hutchpp_grad_values(A, lo, hi, m, ref["Q"], ref["Gp"])
    assert rel_err(g.cpu().numpy(), want) < 1e-9
    dv = _dtheta_values(A)
    th = L.ll_param_grad(h, g, torch.as_tensor(dv).cuda())
    assert th[0] == pytest.approx(float(want @ dv), rel=1e-9)


def test_gmrf_theta_exact_trace_and_derivative_closed_form(L, h):
    """k >= n: the estimate is the exact polynomial trace and d/dtheta approaches
    tr(Q^-1 Adj) = sum_ij (a_i + a_j) / (1 + theta (a_i + a_j))."""
    torch = need_gpu()
    N, theta = 7, -0.24
    A = gmrf_theta(N, theta)
    lo, hi = O.gershgorin(A)
    dA = L.DeviceCSR.from_host(A)
    est = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=90, probes=3 * A.n, seed=1, keep_for_backward=True))
    assert est == pytest.approx(pins.logdet_gmrf_theta(N, theta), rel=1e-9, abs=1e-9)
    g = L.ll_logdet_backward(h, dA, 1.0)
    th = L.ll_param_grad(h, g, torch.as_tensor(_dtheta_values(A)).cuda())
    assert th[0] == pytest.approx(pins.dlogdet_gmrf_theta(N, theta), rel=1e-6)
