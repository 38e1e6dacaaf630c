"""Parity at the workloads' full sizes (needs a GB300).

p(A)V is computed on the GPU for the whole probe block, in the launch shapes of the benchmark
(33 columns as in pass 1, 66 as in pass 2), and sampled columns are recomputed by the oracle one
at a time. Estimates at full size are checked through properties that hold at any size: FP64-class
paths agree with each other, FP32-mixed stays within its tolerance, and the error against the
closed-form log-determinant is within the polynomial and sampling error.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import logdet as O
from oracle import rng as R
from synth import gmrf_batch_params, laplacian_2d, laplacian_3d, matern_2d, matern_2d_derivatives, powerlaw_laplacian
from tests import pins
from tests.gpu_util import TOL, lib, need_gpu, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


@pytest.fixture(scope="module")
def lap3d():
    return laplacian_3d(128, 0.05)


def _sampled_columns(L, h, A, lmin, lmax, degree, V, cols, prec):
    torch = need_gpu()
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    PV = L.ll_apply_poly(h, dA, lmin, lmax, degree, torch.as_tensor(V).cuda(), prec)
    got = PV[:, cols].cpu().numpy()
    want = O.apply_poly(A, V[:, cols], lmin, lmax, degree)
    return got, want


@pytest.mark.parametrize("prec", ["df64", "f32"])
def test_config2_pass1_shape_sampled_columns(L, h, lap3d, prec):
    """128^3 Laplacian + 0.05 I, degree 60, the 33-column Rademacher sketch of seed 1."""
    V = R.rademacher(1, R.STREAM_S, lap3d.n, 33)
    got, want = _sampled_columns(L, h, lap3d, 0.05, 12.05, 60, V, [0, 32], prec)
    assert rel_err(got, want) < TOL[prec]


def test_config2_pass2_shape_sampled_columns(L, h, lap3d):
    """66 columns (the pass-2 width), Gaussian block, degree 60, DF64."""
    V = np.random.default_rng(11).standard_normal((lap3d.n, 66))
    got, want = _sampled_columns(L, h, lap3d, 0.05, 12.05, 60, V, [0, 65], "df64")
    assert rel_err(got, want) < TOL["df64"]


def test_config2_estimates_full_size(L, h, lap3d):
    dA = L.DeviceCSR.from_host(lap3d)
    dA32 = L.DeviceCSR.from_host(lap3d, "f32")
    est = {}
    for prec in ("df64", "f64", "f32"):
        A = dA32 if prec == "f32" else dA
        est[prec] = L.ll_logdet_forward(h, A, 0.05, 12.05, L.options(degree=60, probes=99, seed=1, precision=prec))
    assert abs(est["df64"] - est["f64"]) / abs(est["f64"]) < 1e-10
    assert abs(est["f32"] - est["f64"]) / abs(est["f64"]) < 2e-5
    exact = pins.logdet_laplacian_3d(128, 0.05)
    assert abs(est["df64"] - exact) / exact < 1e-3


def test_config3_matern_full_size(L, h):
    """1024^2 Matérn (13-point stencil), degree 80: sampled columns of p(A)V against the oracle,
    the Gaussian-probe estimate and the (kappa, tau) gradients against the closed forms."""
    torch = need_gpu()
    kappa, tau = 0.3, 1.0
    A = matern_2d(1024, kappa, tau)
    lmax = O.gershgorin(A)[1]
    lmin = tau * kappa ** 4
    V = R.gaussian(0, R.STREAM_S, A.n, 20)
    got, want = _sampled_columns(L, h, A, lmin, lmax, 80, V, [3], "df64")
    assert rel_err(got, want) < TOL["df64"]
    dA = L.DeviceCSR.from_host(A)
    opts = L.options(degree=80, probes=60, seed=0, precision="df64", probe_kind="gaussian", keep_for_backward=True)
    est = L.ll_logdet_forward(h, dA, lmin, lmax, opts)
    assert abs(est - pins.logdet_matern_2d(1024, kappa, tau)) / abs(est) < 1e-3
    g = L.ll_logdet_backward(h, dA, 1.0)
    dk, dt = matern_2d_derivatives(1024, kappa, tau)
    th = L.ll_param_grad(h, g, torch.as_tensor(np.stack([dk, dt])).cuda())
    ex_k, ex_t = pins.dlogdet_matern_2d(1024, kappa, tau)
    assert abs(th[0] - ex_k) / ex_k < 5e-3
    assert abs(th[1] - ex_t) / ex_t < 5e-3


def test_config4_batched_full_size(L, h):
    """All 64 matrices in one batched call; three sampled matrices recomputed one by one."""
    params = gmrf_batch_params(count=64, seed=2)
    mats = [laplacian_2d(side, t) for side, t in params]
    bounds = [(t, 8.0 + t) for _, t in params]
    dm = [L.DeviceCSR.from_host(A) for A in mats]
    est = L.ll_logdet_batched(h, dm, bounds, L.options(probes=30, seed=2, precision="df64"))
    for i in (0, 31, 63):
        lo, hi = bounds[i]
        m = O.degree_from_bounds(lo / O.sigma_of(lo), hi / O.sigma_of(lo))
        single = L.ll_logdet_forward(h, dm[i], lo, hi, L.options(degree=m, probes=30, seed=2 + i, precision="df64"))
        assert est[i] == pytest.approx(single, rel=1e-12)
    exact = np.array([pins.logdet_laplacian_2d(side, t) for side, t in params])
    assert np.median(np.abs(est - exact) / np.abs(exact)) < 5e-3


@pytest.mark.parametrize("prec", ["df64", "f32"])
def test_config5_powerlaw_reduced_size(L, h, prec):
    """Power-law graph Laplacian + 1e-2 I at n = 2^14 (the workload's generator): Gershgorin plus
    20 power iterations for the bounds, degree 150, 120 probes, against the oracle."""
    A = powerlaw_laplacian(1 << 14, seed=3)
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    lo, hi = L.ll_gershgorin(h, L.DeviceCSR.from_host(A))
    lp = L.ll_power_lmax(h, L.DeviceCSR.from_host(A), iters=20, seed=3)
    assert (lo, hi) == O.gershgorin(A)
    assert lp == pytest.approx(O.power_iteration_lmax(A, 20, 3), rel=1e-10)
    lmin, lmax = 0.01, min(hi, 1.05 * lp)
    got = L.ll_logdet_forward(h, dA, lmin, lmax, L.options(degree=150, probes=120, seed=3, precision=prec))
    want = O.logdet_leja(A, lmin, lmax, 150, 120, 3)["estimate"]
    assert abs(got - want) / abs(want) < TOL[prec]
    assert math.isfinite(got)


@pytest.fixture(scope="module")
def lap3d_80():
    return laplacian_3d(80, 0.05)


@pytest.fixture(scope="module")
def oracle_80(lap3d_80):
    cache = {}

    def get(f32: bool):
        if f32 not in cache:
            cache[f32] = O.logdet_leja(lap3d_80, 0.05, 12.05, 20, 99, 4, f32=f32)
        return cache[f32]
    return get


@pytest.mark.parametrize("prec", ["df64", "f64", "f32"])
def test_hutchpp_multi_tile_gram_matches_oracle(L, h, lap3d_80, oracle_80, prec):
    """80^3 Laplacian + 0.05 I (n = 512,000), Hutch++ with k = 33, degree 20: large enough that
    every CTA of the CholeskyQR2 Gram launches sums more than QR_FLUSH = 8 row tiles (13 tiles of
    128 rows per CTA for Y^T Y, 26 of 64 rows for Q^T G) before the running double-float sum and
    the fixed-order reduction of 304 CTA partials. The estimate and G' = (I - Q Q^T) G (unique for
    the span, so compared element by element) against the oracle's Householder path."""
    A = lap3d_80
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    opts = L.options(degree=20, probes=99, seed=4, precision=prec, keep_for_backward=True)
    got = L.ll_logdet_forward(h, dA, 0.05, 12.05, opts)
    ref = oracle_80(prec == "f32")
    assert abs(got - ref["estimate"]) < TOL[prec] * abs(ref["estimate"])
    Q, Gp = (t.cpu().numpy() for t in L.ll_kept_basis(h))
    assert rel_err(Gp, ref["Gp"]) < TOL[prec]
    assert np.max(np.abs(Q.T @ Q - np.eye(33))) < (1e-12 if prec != "f32" else 1e-6)
