"""The banded multi-step kernel (needs a GB300 and the library).

For matrices whose rows hold strictly increasing columns within two of the diagonal, the library
runs up to four Léja steps per launch on row tiles with halos. W_{j+1} and P are then the
one-step kernels' values bit for bit (same per-row arithmetic, same entry order), and the
estimates agree with the oracle at the parity bar.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from synth import CSR, csr_from_dense, laplacian_2d, pentadiagonal
from tests import pins
from tests.gpu_util import TOL, lib, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


def _tridiagonal(n: int, seed: int) -> CSR:
    """SPD tridiagonal: off-diagonals U[-1, 1], diagonal 2.5 + U[0, 1] (diagonally dominant)."""
    rs = np.random.default_rng(seed)
    off = rs.uniform(-1, 1, n - 1)
    diag = 2.5 + rs.uniform(0, 1, n)
    import scipy.sparse as sp
    return CSR.from_scipy(sp.diags([off, diag, off], [-1, 0, 1], format="csr"))


def _apply(L, h, A, lmin, lmax, degree, V, prec, kernel):
    torch = need_gpu()
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    h.set_step_config(kernel, 0, 0)
    try:
        out = L.ll_apply_poly(h, dA, lmin, lmax, degree, torch.as_tensor(V).cuda(), prec)
        info = h.info()
    finally:
        h.set_step_config("auto", 0, 0)
    return out, info


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("n,b,degree", [(2049, 5, 9), (1000, 10, 40), (777, 33, 4), (300, 1, 7), (5, 3, 6), (3, 2, 5)])
def test_band_equals_one_step_kernels_bit_for_bit(L, h, prec, n, b, degree):
    """P = p(A) V on the banded kernel and on the register-gather kernel: identical. Ragged n,
    tiny n, odd widths, degrees that are not multiples of four."""
    A = pentadiagonal(n, seed=n) if n > 4 else _tridiagonal(n, seed=1)
    lo, hi = O.gershgorin(A)
    V = np.random.default_rng(b).standard_normal((A.n, b))
    band, ib = _apply(L, h, A, lo, hi, degree, V, prec, "band")
    ref, ig = _apply(L, h, A, lo, hi, degree, V, prec, "gather")
    assert ib["kernel_pass1"] == L.LL_KERNEL_BAND and ig["kernel_pass1"] == L.LL_KERNEL_GATHER
    assert band.equal(ref)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_band_apply_matches_oracle(L, h, prec):
    A = _tridiagonal(4099, seed=3)
    lo, hi = O.gershgorin(A)
    V = np.random.default_rng(0).standard_normal((A.n, 7))
    got, info = _apply(L, h, A, lo, hi, 25, V, prec, "auto")
    assert info["kernel_pass1"] == L.LL_KERNEL_BAND
    want = O.apply_poly(A, V, lo, hi, 25, f32=(prec == "f32"))
    assert rel_err(got.cpu().numpy(), want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("est", ["hutchpp", "hutchinson"])
def test_band_forward_matches_oracle_and_tma(L, h, prec, est):
    """The pentadiagonal family at n = 3001: the banded kernel under auto, against the oracle and
    against the TMA kernel (the traces are summed in another order)."""
    A = pentadiagonal(3001, seed=5)
    lo, hi = O.gershgorin(A)
    m = 13
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    got = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=m, probes=24, seed=2, precision=prec, estimator=est))
    info = h.info()
    assert info["kernel_pass2"] == L.LL_KERNEL_BAND
    assert est == "hutchinson" or info["kernel_pass1"] == L.LL_KERNEL_BAND
    tma = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=m, probes=24, seed=2, precision=prec, estimator=est,
                                                       step_kernel="tma"))
    assert h.info()["kernel_pass2"] == L.LL_KERNEL_TMA
    assert abs(got - tma) <= 1e-13 * abs(tma)
    f32 = prec == "f32"
    if est == "hutchinson":
        want = O.logdet_hutchinson(A, lo, hi, m, 24, 2, f32=f32)["estimate"]
    else:
        want = O.logdet_leja(A, lo, hi, m, 24, 2, f32=f32)["estimate"]
    assert abs(got - want) / abs(want) < TOL[prec]


def test_band_exact_trace_against_banded_cholesky(L, h):
    """k >= n on the banded kernel: the estimate is the exact polynomial trace, within the
    interpolation error of the banded-Cholesky log-determinant."""
    A = pentadiagonal(60, seed=7)
    lo, hi = O.gershgorin(A)
    dA = L.DeviceCSR.from_host(A)
    got = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=30, probes=180, seed=1))
    assert h.info()["kernel_pass2"] == L.LL_KERNEL_BAND
    assert got == pytest.approx(pins.logdet_banded(A), rel=1e-12)


def test_band_not_taken_for_other_matrices(L, h):
    """Entries farther than two from the diagonal, or a row whose columns are not strictly
    increasing, keep the one-step kernels, with the same results."""
    A = laplacian_2d(20, 0.5)
    V = np.random.default_rng(1).standard_normal((A.n, 4))
    _, info = _apply(L, h, A, 0.5, 8.5, 10, V, "df64", "band")
    assert info["kernel_pass1"] != L.LL_KERNEL_BAND
    B = _tridiagonal(200, seed=2)
    rp, ci, va = B.rowptr.copy(), B.colind.copy(), B.values.copy()
    a = rp[100]
    ci[a], ci[a + 1] = ci[a + 1], ci[a]          # row 100: columns out of order
    va[a], va[a + 1] = va[a + 1], va[a]
    Bu = CSR(B.n, rp, ci, va)
    W = np.random.default_rng(3).standard_normal((B.n, 3))
    got, info = _apply(L, h, Bu, *O.gershgorin(B), 12, W, "df64", "auto")
    assert info["kernel_pass1"] != L.LL_KERNEL_BAND
    want = O.apply_poly(B, W, *O.gershgorin(B), 12)
    assert rel_err(got.cpu().numpy(), want) < 1e-10


def test_backward_qr_uses_the_kept_matrix_band_choice(L, h):
    """The through-QR adjoint's pass-1 sweep runs on the kept forward's matrix: a call on another
    matrix in between (banded or not) must not change the kernel it takes."""
    torch = need_gpu()
    from synth import random_spd
    for A, other in ((random_spd(600, seed=9), pentadiagonal(500, seed=1)), (pentadiagonal(700, seed=2), random_spd(400, seed=3))):
        lo, hi = O.gershgorin(A)
        lmin = max(lo, 0.05)
        dA = L.DeviceCSR.from_host(A)
        L.ll_logdet_forward(h, dA, lmin, hi, L.options(degree=15, probes=12, seed=4, keep_for_backward=True))
        olo, ohi = O.gershgorin(other)
        V = torch.as_tensor(np.random.default_rng(0).standard_normal((other.n, 3))).cuda()
        L.ll_apply_poly(h, L.DeviceCSR.from_host(other), max(olo, 0.05), ohi, 5, V, "df64")
        g = L.ll_logdet_backward(h, dA, 1.0, through_qr=True).cpu().numpy()
        S, G = O.make_probes(A.n, 4, 4)
        want = O.hutchpp_full_grad_values(A, lmin, hi, 15, S, G)
        assert rel_err(g, want) < 1e-9
