"""GPU-vs-oracle parity through the C ABI (needs a GB300 and the built library).

Bars: integer/index work and Rademacher probes bit-exact; FP64-class paths (f64, df64) within a
relative 1e-10 of the oracle, FP32-mixed within 2e-5, measured as max-norm relative error of the
block (or relative error of a scalar).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import logdet as O
from oracle import rng as ORNG
from synth import CSR, diagonal, laplacian_2d, laplacian_3d, matern_2d, powerlaw_laplacian, random_spd
from tests.gpu_util import TOL, lib, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


# ---------------------------------------------------------------------------- probes and bounds

@pytest.mark.parametrize("kind", ["rademacher", "gaussian"])
def test_probes_match_oracle(L, h, kind):
    n, cols = 10007, 13
    for stream_id in (0, 1, 2):
        got = L.ll_probes(h, kind, 12345, stream_id, n, cols).cpu().numpy()
        want = ORNG.probes(kind, 12345, stream_id, n, cols)
        if kind == "rademacher":
            assert np.array_equal(got, want)
        else:
            assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("make", [lambda: laplacian_2d(37, 0.1), lambda: random_spd(3001, seed=3, empty_rows=5, dense_row=True),
                                  lambda: matern_2d(20, 0.3, 1.0)])
def test_gershgorin_matches_oracle(L, h, make):
    A = make()
    got = L.ll_gershgorin(h, L.DeviceCSR.from_host(A))
    want = O.gershgorin(A)
    assert got == want


def test_power_iteration(L, h):
    A = random_spd(5000, seed=7)
    got = L.ll_power_lmax(h, L.DeviceCSR.from_host(A), iters=20, seed=3)
    want = O.power_iteration_lmax(A, iters=20, seed=3)
    assert got == pytest.approx(want, rel=1e-12)


# ------------------------------------------------------------------------------ p(A) V (Alg. 2)

def _apply_case(L, h, A, lmin, lmax, degree, b, prec, seed=0):
    torch = need_gpu()
    V = np.random.default_rng(seed).standard_normal((A.n, b))
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    got = L.ll_apply_poly(h, dA, lmin, lmax, degree, torch.as_tensor(V).cuda(), prec).cpu().numpy()
    want = O.apply_poly(A, V, lmin, lmax, degree)
    return got, want


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("b", [1, 3, 10, 33, 66])
def test_apply_poly_random_spd(L, h, prec, b):
    # ragged n, empty rows (diagonal only) and one dense row
    A = random_spd(2111, nnz_per_row=7, seed=b, empty_rows=4, dense_row=True)
    lam_lo, lam_hi = O.gershgorin(A)
    lmin = max(lam_lo, 0.05)
    got, want = _apply_case(L, h, A, lmin, lam_hi, 25, b, prec)
    assert rel_err(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("degree", [0, 1, 2, 39])
def test_apply_poly_degrees(L, h, prec, degree):
    A = laplacian_2d(41, 0.1)
    got, want = _apply_case(L, h, A, 0.1, 8.1, degree, 10, prec)
    assert rel_err(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_apply_poly_3d_and_matern(L, h, prec):
    A = laplacian_3d(13, 0.05)
    got, want = _apply_case(L, h, A, 0.05, 12.05, 60, 7, prec)
    assert rel_err(got, want) < TOL[prec]
    M = matern_2d(24, 0.3, 1.0)
    lo, hi = O.gershgorin(M)
    got, want = _apply_case(L, h, M, 0.0081, hi, 40, 5, prec)
    assert rel_err(got, want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_apply_poly_powerlaw_long_rows(L, h, prec):
    """Irregular rows, some longer than a shared-memory tile holds (global-memory fallback)."""
    A = powerlaw_laplacian(1 << 13, seed=3)
    lo, hi = O.gershgorin(A)
    got, want = _apply_case(L, h, A, 0.01, hi, 30, 12, prec)
    assert rel_err(got, want) < TOL[prec]


def test_apply_poly_diagonal_matrix(L, h):
    d = np.linspace(0.3, 5.0, 777)
    A = diagonal(d)
    got, want = _apply_case(L, h, A, 0.3, 5.0, 30, 4, "df64")
    assert rel_err(got, want) < 1e-10


# -------------------------------------------------------------------------- estimator (Alg. 3)

def _forward(L, h, A, lmin, lmax, degree, probes, seed, prec, kind="rademacher", keep=False):
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    opts = L.options(degree=degree, probes=probes, seed=seed, precision=prec, probe_kind=kind, keep_for_backward=keep)
    return L.ll_logdet_forward(h, dA, lmin, lmax, opts)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_forward_config1_matches_oracle(L, h, prec):
    """2-D Laplacian + 0.1 I (100 x 100), bounds [0.1, 8.1], 40 Léja points, 30 Rademacher
    probes from seed 0."""
    A = laplacian_2d(100, 0.1)
    got = _forward(L, h, A, 0.1, 8.1, 39, 30, 0, prec)
    want = O.logdet_leja(A, 0.1, 8.1, 39, 30, 0)["estimate"]
    assert abs(got - want) / abs(want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_forward_gaussian_matern(L, h, prec):
    A = matern_2d(32, 0.3, 1.0)
    lo, hi = O.gershgorin(A)
    got = _forward(L, h, A, 0.0081, hi, 50, 12, 5, prec, kind="gaussian")
    want = O.logdet_leja(A, 0.0081, hi, 50, 12, 5, kind="gaussian")["estimate"]
    assert abs(got - want) / abs(want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_forward_kept_basis(L, h, prec):
    """G' = (I - Q Q^T) G is unique for a given span, so it is compared element by element;
    Q is compared through its projector."""
    A = random_spd(1500, seed=2)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    dA = L.DeviceCSR.from_host(A)
    opts = L.options(degree=20, probes=24, seed=9, precision=prec, keep_for_backward=True)
    L.ll_logdet_forward(h, dA, lmin, hi, opts)
    Q, Gp = (t.cpu().numpy() for t in L.ll_kept_basis(h))
    ref = O.logdet_leja(A, lmin, hi, 20, 24, 9)
    assert rel_err(Gp, ref["Gp"]) < 1e-10
    Qo = ref["Q"]
    assert np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) < 1e-12
    assert np.max(np.abs(Q @ (Q.T @ Qo) - Qo)) < 1e-10


def test_forward_probes_ge_n(L, h):
    """k >= n: the sketch spans R^n and the estimate is the exact polynomial trace."""
    A = random_spd(7, seed=1)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    got = _forward(L, h, A, lmin, hi, 15, 30, 4, "df64")
    want = O.logdet_leja(A, lmin, hi, 15, 30, 4)["estimate"]
    assert abs(got - want) < 1e-10 * abs(want) + 1e-12


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_forward_pentadiagonal_matches_oracle(L, h, prec):
    """Section 5.1's synthetic pentadiagonal family (n = 4000, Gershgorin bounds, degree from the
    bounds, 30 Rademacher probes): the GPU estimate matches the oracle on the same probes."""
    from synth import pentadiagonal
    A = pentadiagonal(4000, seed=4)
    lo, hi = O.gershgorin(A)
    m = O.degree_from_bounds(lo, hi)   # sigma = 1: lambda_min >= 1
    got = _forward(L, h, A, lo, hi, m, 30, 1, prec)
    want = O.logdet_leja(A, lo, hi, m, 30, 1, f32=(prec == "f32"))["estimate"]
    assert abs(got - want) / abs(want) < TOL[prec]


def test_forward_pentadiagonal_exact_trace_equals_banded_cholesky(L, h):
    """With as many sketch columns as rows (the Q = I branch) the GPU estimate is the exact
    polynomial trace, which on this spectrum equals the banded-Cholesky log-determinant."""
    from synth import pentadiagonal
    from tests import pins
    A = pentadiagonal(90, seed=2)
    lo, hi = O.gershgorin(A)
    m = O.degree_from_bounds(lo, hi)
    got = _forward(L, h, A, lo, hi, m, 270, 5, "df64")
    assert got == pytest.approx(pins.logdet_banded(A), rel=1e-11)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("kind", ["rademacher", "gaussian"])
def test_forward_hutchinson_matches_oracle(L, h, prec, kind):
    """Plain Hutchinson (Eq. Léja8, `estimator="hutchinson"`): no sketch and no QR; the GPU
    estimate over 25 probes of the G stream matches the oracle's."""
    A = matern_2d(40, 0.3, 1.0)
    lo, hi = O.gershgorin(A)
    lmin = 0.0081
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    got = L.ll_logdet_forward(h, dA, lmin, hi, L.options(degree=50, probes=25, seed=2, precision=prec, probe_kind=kind,
                                                         estimator="hutchinson"))
    info = h.info()
    want = O.logdet_hutchinson(A, lmin, hi, 50, 25, 2, kind=kind, f32=(prec == "f32"))["estimate"]
    assert abs(got - want) / abs(want) < TOL[prec]
    assert info["k"] == 0 and info["ms_qr"] < 0.05


def test_forward_hutchinson_exact_on_diagonal_and_limits(L, h):
    """Rademacher Hutchinson is exact on a diagonal matrix for any probe count; probe counts
    need not be multiples of 3; more than 192 probes are refused, and the batched call runs
    Hutch++ only."""
    dvals = np.linspace(0.3, 5.0, 333)
    A = diagonal(dvals)
    dA = L.DeviceCSR.from_host(A)
    got = L.ll_logdet_forward(h, dA, 0.3, 5.0, L.options(degree=30, probes=4, seed=9, estimator="hutchinson"))
    want = O.logdet_hutchinson(A, 0.3, 5.0, 30, 4, 9)["estimate"]
    assert got == pytest.approx(want, rel=1e-10)
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_forward(h, dA, 0.3, 5.0, L.options(degree=30, probes=193, estimator="hutchinson"))
    assert ei.value.name == "LL_ERR_UNSUPPORTED"
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_batched(h, [dA], [(0.3, 5.0)], L.options(probes=30, estimator="hutchinson"))
    assert ei.value.name == "LL_ERR_UNSUPPORTED"


def test_forward_empty_matrix(L, h):
    A = CSR(n=0, rowptr=np.zeros(1, dtype=np.int32), colind=np.zeros(0, dtype=np.int32), values=np.zeros(0))
    torch = need_gpu()
    dA = L.DeviceCSR(n=0, rowptr=torch.zeros(1, dtype=torch.int32, device="cuda"),
                     colind=torch.zeros(0, dtype=torch.int32, device="cuda"),
                     values=torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert L.ll_logdet_forward(h, dA, 0.5, 2.0, L.options()) == 0.0
    del A


def test_forward_degenerate_scaled_identity(L, h):
    """A = sigma I with lmin = sigma: A/sigma = I and p(I) = log 1 = 0, so the sketch is pure
    rounding noise; any orthonormal basis of it gives the exact answer n log sigma."""
    A = diagonal(np.full(500, 0.5))
    got = _forward(L, h, A, 0.5, 2.0, 10, 9, 0, "df64")
    want = O.logdet_leja(A, 0.5, 2.0, 10, 9, 0)["estimate"]
    assert got == pytest.approx(500 * math.log(0.5), rel=1e-12)
    assert got == pytest.approx(want, rel=1e-12)


def test_forward_rank_deficient_sketch_is_reported(L, h):
    """Two identical sketch columns make Y rank-deficient: CholeskyQR reports a breakdown
    (the oracle's Householder QR would still return some basis)."""
    n, k = 3, 2
    seed = next(s for s in range(1000)
                if np.array_equal(*ORNG.rademacher(s, 0, n, k).T) and not np.array_equal(*ORNG.rademacher(s, 1, n, k).T))
    A = random_spd(n, seed=1)
    lo, hi = O.gershgorin(A)
    with pytest.raises(L.LejaError) as ei:
        _forward(L, h, A, max(lo, 0.05), hi, 8, 3 * k, seed, "df64")
    assert ei.value.name == "LL_ERR_QR_BREAKDOWN"


def test_error_codes(L, h):
    torch = need_gpu()
    A = laplacian_2d(10, 0.1)
    dA = L.DeviceCSR.from_host(A)
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_forward(h, dA, 0.0, 8.1, L.options())
    assert ei.value.name == "LL_ERR_BAD_BOUNDS"
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_forward(h, dA, 9.0, 8.1, L.options())
    assert ei.value.name == "LL_ERR_BAD_BOUNDS"
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_forward(h, dA, 0.1, 8.1, L.options(probes=10))
    assert ei.value.name == "LL_ERR_INVALID_ARG"
    bad = L.DeviceCSR(n=A.n, rowptr=dA.rowptr, colind=dA.colind.clone(), values=dA.values)
    bad.colind[5] = A.n + 3
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_forward(h, bad, 0.1, 8.1, L.options())
    assert ei.value.name == "LL_ERR_BAD_CSR"
    bad2 = L.DeviceCSR(n=A.n, rowptr=dA.rowptr.clone(), colind=dA.colind, values=dA.values)
    bad2.rowptr[3] = bad2.rowptr[4] + 1
    with pytest.raises(L.LejaError) as ei:
        L.ll_gershgorin(h, bad2)
    assert ei.value.name == "LL_ERR_BAD_CSR"
    # the handle stays usable after errors
    est = L.ll_logdet_forward(h, dA, 0.1, 8.1, L.options(degree=10, probes=6))
    assert math.isfinite(est)
    del torch


def test_forward_host_path_matches_device_path(L, h):
    A = laplacian_2d(60, 0.1)
    opts = L.options(degree=30, probes=15, seed=2, precision="df64")
    e_dev = L.ll_logdet_forward(h, L.DeviceCSR.from_host(A), 0.1, 8.1, opts)
    e_host = L.ll_logdet_forward_host(h, A, 0.1, 8.1, opts)
    assert e_dev == e_host


def test_trim_workspace_frees_memory_and_the_next_call_reallocates(L):
    """ll_trim_workspace frees the handle's blocks (the device's free memory grows back), drops the
    kept forward (the backward refuses), and the next forward gives the same estimate."""
    torch = need_gpu()
    from synth import laplacian_3d
    A = laplacian_3d(64, 0.05)
    dA = L.DeviceCSR.from_host(A)
    h = L.Handle()
    o = L.options(degree=20, probes=30, seed=3, keep_for_backward=True, step_kernel="tma", qr_gram="dfloat")
    e1 = L.ll_logdet_forward(h, dA, 0.05, 12.05, o)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    h.trim()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after > free_before + (64 << 20)
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_backward(h, dA, 1.0)
    assert ei.value.name == "LL_ERR_NO_FORWARD"
    e2 = L.ll_logdet_forward(h, dA, 0.05, 12.05, o)
    assert e1 == e2
