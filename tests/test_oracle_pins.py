"""Pins of the oracle against the paper and the mathematics (CPU only).

Each oracle function is checked against something other than itself: hand-derived values,
published known-answer outputs, a high-precision textbook recurrence, SciPy's barycentric
interpolation, dense eigendecompositions, closed-form log-determinants and finite differences.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import divdiff, leja, logdet, rng
from synth import (csr_from_dense, diagonal, laplacian_2d, laplacian_3d, matern_2d,
                   matern_2d_derivatives, random_spd)
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------------------------ Léja points

def test_leja_prefix_hand_derived():
    want = [float(r[0]) for r in _golden_rows("leja_prefix.txt")]
    got = leja.fast_leja_points(len(want))
    assert got.tolist() == want


def test_leja_matches_exact_rational_construction():
    """Fast Léja points by exact rational arithmetic (no rounding anywhere; ties -> smaller x)
    agree with the FP64 construction on a 60-point prefix."""
    count = 60
    pts = [Fraction(2), Fraction(-2)]
    while len(pts) < count:
        srt = sorted(pts)
        best, best_x = None, None
        for a, b in zip(srt[:-1], srt[1:]):
            x = (a + b) / 2
            s = Fraction(1)
            for p in pts:
                s *= abs(x - p)
            if best is None or s > best:
                best, best_x = s, x
        pts.append(best_x)
    got = leja.fast_leja_points(count)
    assert got.tolist() == [float(p) for p in pts]


def test_leja_greedy_property_against_grid():
    """Each fast Léja point nearly maximises prod |x - xi_k| over a fine grid of [-2, 2]
    (the continuous definition, Eq. Léja5): within a factor 0.5, and the points are distinct."""
    xi = leja.fast_leja_points(80)
    assert len(set(xi.tolist())) == 80
    assert np.all(np.abs(xi) <= 2.0)
    grid = np.linspace(-2, 2, 200001)
    logs = np.zeros_like(grid)
    for j in range(1, 80):
        logs += np.log(np.abs(grid - xi[j - 1]) + 1e-300)
        val = np.sum(np.log(np.abs(xi[j] - xi[:j])))
        assert val >= logs.max() + math.log(0.5)


# ------------------------------------------------------------------------ divided differences

@pytest.mark.parametrize("lmin,lmax,m", [
    (0.1, 8.1, 39),          # 2-D Laplacian + 0.1 I, before sigma-normalisation
    (1.0, 81.0, 39),         # the same interval after sigma-normalisation
    (1.0, 241.0, 60),        # 3-D Laplacian + 0.05 I
    (1.0, 241.0, 120),
    (1.0, 8080.0, 80),       # Matérn tau (kappa^2 I + L)^2 with kappa = 0.3
    (2.0, 3.0, 10),
])
def test_divided_differences_vs_high_precision_recurrence(lmin, lmax, m):
    xi = leja.fast_leja_points(m + 1)
    c, g = (lmin + lmax) / 2, (lmax - lmin) / 4
    d, p = divdiff.divided_differences(xi, c, g)
    ref = pins.hp_scaled_divided_differences(lmin, lmax, xi)
    assert np.max(np.abs(d - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_divided_differences_two_point_closed_form():
    lmin, lmax = 0.3, 7.0
    xi = leja.fast_leja_points(2)          # z_0 = lmax, z_1 = lmin
    c, g = (lmin + lmax) / 2, (lmax - lmin) / 4
    d, _ = divdiff.divided_differences(xi, c, g)
    assert d[0] == pytest.approx(math.log(lmax), rel=1e-15)
    assert d[1] == pytest.approx(g * (math.log(lmin) - math.log(lmax)) / (lmin - lmax), rel=1e-13)


def test_divided_differences_interpolate_log_at_nodes():
    lmin, lmax, m = 0.05, 12.05, 60
    xi = leja.fast_leja_points(m + 1)
    c, g = (lmin + lmax) / 2, (lmax - lmin) / 4
    d, _ = divdiff.divided_differences(xi, c, g)
    for i in range(0, m + 1, 7):
        z = c + g * xi[i]
        assert pins.newton_value_hp(d, xi, lmin, lmax, z) == pytest.approx(math.log(z), rel=1e-12, abs=1e-12)


def test_divided_differences_independent_of_s():
    """log(Q_m) e_1 does not depend on s_val (only the series' convergence does): a dropped
    log(s) term or a wrong Taylor sign would make the two disagree."""
    lmin, lmax, m = 1.0, 50.0, 40
    xi = leja.fast_leja_points(m + 1)
    c, g = (lmin + lmax) / 2, (lmax - lmin) / 4
    d1, _ = divdiff.divided_differences(xi, c, g, s=c)
    d2, _ = divdiff.divided_differences(xi, c, g, s=0.7 * lmax)
    assert np.max(np.abs(d1 - d2)) <= 1e-12 * np.max(np.abs(d1))


def test_divided_differences_sigma_invariance():
    """Scaling the interval by 1/sigma leaves d_j (j >= 1) unchanged and shifts d_0 by -log sigma."""
    lmin, lmax, m = 0.1, 8.1, 39
    sigma = logdet.sigma_of(lmin)
    _, _, _, d1, _ = logdet.newton_leja_setup(lmin, lmax, m)
    _, _, _, d2, _ = logdet.newton_leja_setup(lmin / sigma, lmax / sigma, m)
    assert d2[0] == pytest.approx(d1[0] - math.log(sigma), rel=1e-13)
    assert np.max(np.abs(d1[1:] - d2[1:])) <= 1e-12 * np.max(np.abs(d1))


def test_divided_differences_nonconvergence_is_an_error():
    xi = leja.fast_leja_points(21)
    with pytest.raises(divdiff.DividedDifferenceError):
        divdiff.divided_differences(xi, 5.0, 2.4, s=5.0, max_terms=50)


def test_taylor_term_counts_grow_with_condition_number():
    # s = c gives |z/s - 1| <= (k-1)/(k+1); the term counts grow with the condition number
    _, _, _, _, p1 = logdet.newton_leja_setup(1.0, 81.0, 39)
    _, _, _, _, p3 = logdet.newton_leja_setup(1.0, 8080.0, 80)
    assert 500 < p1 < 5000
    assert 20000 < p3 < 500000


# --------------------------------------------------------------------------------------- probes

def test_splitmix64_known_answers():
    golden = 0x9E3779B97F4A7C15
    for seed, idx, val in _golden_rows("splitmix64_kat.txt"):
        state = (int(seed) + (int(idx) - 1) * golden) % 2 ** 64
        got = int(rng.mix(np.array([state], dtype=np.uint64))[0])
        assert got == int(val, 16)


def test_probe_counter_layout():
    # x[row, col] for stream s is mix(seed ^ mix(s<<56 | col<<32 | row))
    x = rng.raw_bits(7, 1, 5, 3)
    for r in range(5):
        for c in range(3):
            ctr = (1 << 56) | (c << 32) | r
            inner = int(rng.mix(np.array([ctr], dtype=np.uint64))[0])
            assert int(x[r, c]) == int(rng.mix(np.array([7 ^ inner], dtype=np.uint64))[0])


def test_rademacher_statistics():
    S = rng.rademacher(0, 0, 200000, 4)
    assert set(np.unique(S).tolist()) == {-1.0, 1.0}
    assert np.all(np.abs(S.mean(axis=0)) < 5 / math.sqrt(200000))
    # different columns / streams / seeds are uncorrelated
    G = rng.rademacher(0, 1, 200000, 4)
    assert abs(np.mean(S[:, 0] * S[:, 1])) < 5 / math.sqrt(200000)
    assert abs(np.mean(S[:, 0] * G[:, 0])) < 5 / math.sqrt(200000)
    assert abs(np.mean(S[:, 0] * rng.rademacher(1, 0, 200000, 1)[:, 0])) < 5 / math.sqrt(200000)


def test_gaussian_statistics():
    g = rng.gaussian(3, 0, 400000, 1)[:, 0]
    assert abs(g.mean()) < 5 / math.sqrt(400000)
    assert abs(g.var() - 1.0) < 0.02
    assert abs(np.mean(g ** 4) - 3.0) < 0.1        # Gaussian kurtosis
    assert np.all(np.isfinite(g))


# ------------------------------------------------------------------------------ p(A)V (Alg. 2)

def test_apply_poly_diagonal_matrix_equals_scalar_interpolant():
    n, lmin, lmax, m = 300, 0.2, 9.0, 45
    dvals = np.linspace(lmin, lmax, n) ** 1.0
    A = diagonal(dvals)
    V = rng.rademacher(1, 0, n, 3)
    P = logdet.apply_poly(A, V, lmin, lmax, m)
    p = pins.interpolant(lmin, lmax, leja.fast_leja_points(m + 1))
    ref = p(dvals)[:, None] * V
    assert np.max(np.abs(P - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("seed", [0, 1])
def test_apply_poly_dense_eigendecomposition(seed):
    A = random_spd(150, nnz_per_row=6, seed=seed, empty_rows=3, dense_row=(seed == 1))
    Ad = A.to_scipy().toarray()
    lam = np.linalg.eigvalsh(Ad)
    lmin, lmax = 0.9 * lam[0], 1.1 * lam[-1]
    m = 50
    V = np.random.default_rng(seed).standard_normal((A.n, 4))
    P = logdet.apply_poly(A, V, lmin, lmax, m)
    p = pins.interpolant(lmin, lmax, leja.fast_leja_points(m + 1))
    ref = pins.dense_matrix_function(Ad, p) @ V
    assert np.max(np.abs(P - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_apply_poly_converges_to_log():
    """Proposition 3.1: the error of p_m(A)v against log(A)v decays geometrically."""
    A = laplacian_2d(12, 0.5)
    Ad = A.to_scipy().toarray()
    lmin, lmax = logdet.gershgorin(A)
    V = rng.rademacher(0, 0, A.n, 1)
    ref = pins.dense_matrix_function(Ad, np.log) @ V
    errs = [np.max(np.abs(logdet.apply_poly(A, V, lmin, lmax, m) - ref)) for m in (10, 20, 40, 80)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    kappa = lmax / lmin
    rho = (math.sqrt(kappa) + 1) / (math.sqrt(kappa) - 1)
    assert errs[3] < 50 * rho ** -80 * np.max(np.abs(ref)) + 1e-12


def test_apply_poly_fp32_mode_stays_close():
    A = laplacian_2d(20, 0.1)
    V = rng.rademacher(0, 0, A.n, 2)
    P64 = logdet.apply_poly(A, V, 0.1, 8.1, 39)
    P32 = logdet.apply_poly(A, V, 0.1, 8.1, 39, f32=True)
    err = np.max(np.abs(P64 - P32)) / np.max(np.abs(P64))
    assert 1e-9 < err < 2e-5


# --------------------------------------------------------------------------- bounds and sigma

def test_gershgorin_laplacian_closed_form():
    lo, hi = logdet.gershgorin(laplacian_2d(30, 0.25))
    assert lo == pytest.approx(0.25, abs=1e-14) and hi == pytest.approx(8.25, rel=1e-15)
    lo, hi = logdet.gershgorin(laplacian_3d(9, 0.05))
    assert lo == pytest.approx(0.05, abs=1e-14) and hi == pytest.approx(12.05, rel=1e-15)


def test_gershgorin_contains_spectrum():
    for seed in range(3):
        A = random_spd(120, seed=seed, dense_row=True)
        lam = np.linalg.eigvalsh(A.to_scipy().toarray())
        lo, hi = logdet.gershgorin(A)
        assert lo <= lam[0] + 1e-12 and lam[-1] <= hi + 1e-12
    # hand-made 2x2: [[2, -3], [-3, 5]] -> rows give [-1, 5] and [2, 8]
    lo, hi = logdet.gershgorin(csr_from_dense(np.array([[2.0, -3.0], [-3.0, 5.0]])))
    assert (lo, hi) == (-1.0, 8.0)


def test_power_iteration_bounds_lmax():
    A = random_spd(200, seed=4)
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    lp = logdet.power_iteration_lmax(A, iters=20, seed=3)
    assert lp <= lam[-1] * (1 + 1e-12)
    assert lp >= 0.8 * lam[-1]


def _power_closed_form(a: np.ndarray, c: np.ndarray, k: int) -> float:
    # A = U diag(a) U^T and c = U^T r for the start vector r: after k normalised steps
    # v_k = A^k r / ||A^k r||, so v_k^T A v_k = sum a_i^(2k+1) c_i^2 / sum a_i^(2k) c_i^2
    w = c * c
    return float(np.sum(a ** (2 * k + 1) * w) / np.sum(a ** (2 * k) * w))


@pytest.mark.parametrize("k", [0, 1, 3, 20])
def test_power_iteration_closed_form_diagonal(k):
    # diagonal A: U = I, and the Rademacher start vector has r_i^2 = 1, so the Rayleigh quotient
    # after k steps is sum a^(2k+1) / sum a^(2k) -- not ||A v_k||, and a different k gives a
    # different value (the spread of a keeps the iteration far from converged)
    a = np.linspace(1.0, 2.0, 50)
    got = logdet.power_iteration_lmax(diagonal(a), iters=k, seed=5)
    assert got == pytest.approx(_power_closed_form(a, np.ones_like(a), k), rel=1e-13)
    if k > 0:
        assert abs(got - _power_closed_form(a, np.ones_like(a), k - 1)) > 1e-6
        assert abs(got - _power_closed_form(a, np.ones_like(a), k + 1)) > 1e-6


@pytest.mark.parametrize("k", [1, 4, 20])
def test_power_iteration_closed_form_reflected(k):
    # A = H diag(a) H with the Householder reflector H = I - 2 u u^T / u^T u (H = H^T = H^-1):
    # c = H r depends on the signs of the start vector, so the value pins the generator stream
    # (LL_STREAM_POWER = 2) and the seed as well as the iteration
    n = 40
    a = np.linspace(0.5, 3.0, n)
    u = np.cos(np.arange(n) * 0.7) + 0.3
    H = np.eye(n) - 2.0 * np.outer(u, u) / (u @ u)
    A = csr_from_dense(H @ np.diag(a) @ H)
    seed = 11
    r = rng.rademacher(seed, rng.STREAM_POWER, n, 1)[:, 0]
    got = logdet.power_iteration_lmax(A, iters=k, seed=seed)
    assert got == pytest.approx(_power_closed_form(a, H @ r, k), rel=1e-12)
    for stream in (rng.STREAM_S, rng.STREAM_G):
        r_other = rng.rademacher(seed, stream, n, 1)[:, 0]
        assert abs(got - _power_closed_form(a, H @ r_other, k)) > 1e-8


def test_sigma_rule():
    assert logdet.sigma_of(0.1) == 0.1
    assert logdet.sigma_of(2.0) == 1.0
    with pytest.raises(ValueError):
        logdet.sigma_of(0.0)
    with pytest.raises(ValueError):
        logdet.sigma_of(-1.0)


def test_degree_from_bounds():
    assert logdet.degree_from_bounds(1.0, 9.0) == math.ceil(math.log(1e6) / math.log(2.0))
    assert logdet.degree_from_bounds(1.0, 1e9) == 250
    assert logdet.degree_from_bounds(1.0, 1.0 + 1e-9) == 10
    assert logdet.degree_from_bounds(1.0, 1.5) == 10


# ---------------------------------------------------------------------------- Hutch++ (Alg. 3)

def test_hutchpp_with_k_ge_n_is_the_exact_polynomial_trace():
    """With as many sketch columns as rows, Q spans R^n, the residual part vanishes and the
    estimate is n log sigma + tr p(A / sigma) = sum_i p(lambda_i) exactly."""
    A = random_spd(40, seed=5)
    Ad = A.to_scipy().toarray()
    lam = np.linalg.eigvalsh(Ad)
    lmin, lmax = 0.9 * lam[0], 1.1 * lam[-1]
    m = 30
    S, G = logdet.make_probes(A.n, 40, seed=2)
    r = logdet.hutchpp_logdet(A, lmin, lmax, m, S, G)
    sigma = logdet.sigma_of(lmin)
    p = pins.interpolant(lmin / sigma, lmax / sigma, leja.fast_leja_points(m + 1))
    ref = A.n * math.log(sigma) + float(np.sum(p(lam / sigma)))
    assert r["estimate"] == pytest.approx(ref, rel=1e-11)
    assert abs(r["trace_res"]) < 1e-10


@pytest.mark.parametrize("lscale", [0.02, 3.0])   # sigma < 1 and sigma = 1
def test_hutchpp_matches_dense_route(lscale):
    """Algorithm 3 evaluated through a dense F = p(A/sigma) and an SVD-based orthonormal basis
    (scipy.linalg.orth) instead of the recurrence and Householder QR."""
    from scipy.linalg import orth
    A0 = random_spd(90, seed=6)
    A = csr_from_dense(A0.to_scipy().toarray() * lscale)
    Ad = A.to_scipy().toarray()
    lam = np.linalg.eigvalsh(Ad)
    lmin, lmax = 0.9 * lam[0], 1.1 * lam[-1]
    m, k = 35, 8
    S, G = logdet.make_probes(A.n, k, seed=11)
    r = logdet.hutchpp_logdet(A, lmin, lmax, m, S, G)
    sigma = logdet.sigma_of(lmin)
    p = pins.interpolant(lmin / sigma, lmax / sigma, leja.fast_leja_points(m + 1))
    F = pins.dense_matrix_function(Ad / sigma, p)
    Q = orth(F @ S)
    Gp = G - Q @ (Q.T @ G)
    ref = A.n * math.log(sigma) + np.trace(Q.T @ F @ Q) + np.trace(Gp.T @ F @ Gp) / k
    assert r["estimate"] == pytest.approx(ref, rel=1e-10)


def test_hutchpp_config1_against_closed_form():
    """2-D Laplacian + 0.1 I on 100 x 100, bounds [0.1, 8.1], 40 Léja points, 30 Rademacher
    probes from seed 0: the estimate is close to the closed-form log-determinant."""
    A = laplacian_2d(100, 0.1)
    exact = pins.logdet_laplacian_2d(100, 0.1)
    assert exact == pytest.approx(12232.673634578276, rel=1e-14)
    r = logdet.logdet_leja(A, 0.1, 8.1, 39, 30, 0)
    assert abs(r["estimate"] - exact) / exact < 5e-3


def test_polynomial_bias_config1():
    """The degree-39 interpolant's exact trace differs from the log-determinant by ~4e-7."""
    N, shift, m = 100, 0.1, 39
    mu = pins.lap_eigs_1d(N)
    lam = (mu[:, None] + mu[None, :] + shift).ravel()
    sigma = logdet.sigma_of(0.1)
    p = pins.interpolant(0.1 / sigma, 8.1 / sigma, leja.fast_leja_points(m + 1))
    tr = N * N * math.log(sigma) + math.fsum(p(lam / sigma))
    exact = pins.logdet_laplacian_2d(N, shift)
    assert 1e-8 < abs(tr - exact) / exact < 1e-5


def test_matern_closed_form_matches_dense():
    A = matern_2d(8, 0.3, 1.7)
    sign, ld = np.linalg.slogdet(A.to_scipy().toarray())
    assert sign > 0 and ld == pytest.approx(pins.logdet_matern_2d(8, 0.3, 1.7), rel=1e-12)
    A3 = laplacian_3d(6, 0.05)
    sign, ld = np.linalg.slogdet(A3.to_scipy().toarray())
    assert ld == pytest.approx(pins.logdet_laplacian_3d(6, 0.05), rel=1e-12)


# ----------------------------------------------------------------------------------- gradients

def _fd_check(A, lmin, lmax, m, k, seed, entries, h=1e-6):
    S, G = logdet.make_probes(A.n, k, seed)
    r = logdet.hutchpp_logdet(A, lmin, lmax, m, S, G)
    g = logdet.hutchpp_grad_values(A, lmin, lmax, m, r["Q"], r["Gp"])
    for e in entries:
        vp = A.values.copy(); vp[e] += h
        vm = A.values.copy(); vm[e] -= h
        fd = (logdet.frozen_estimate(A, vp, lmin, lmax, m, r["Q"], r["Gp"])
              - logdet.frozen_estimate(A, vm, lmin, lmax, m, r["Q"], r["Gp"])) / (2 * h)
        assert g[e] == pytest.approx(fd, rel=2e-5, abs=1e-7)
    return g


def test_grad_values_finite_differences_symmetric():
    A = random_spd(60, seed=8)
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    _fd_check(A, 0.9 * lam[0], 1.1 * lam[-1], 25, 5, 3, entries=[0, 7, 33, A.nnz // 2, A.nnz - 1])


def test_grad_values_finite_differences_nonsymmetric():
    """The adjoint uses (B - xi I)^T; a non-symmetric matrix catches a transposed operand."""
    rs = np.random.default_rng(9)
    n = 30
    M = np.diag(rs.uniform(4, 6, n)) + (rs.random((n, n)) < 0.15) * rs.uniform(-0.3, 0.5, (n, n))
    A = csr_from_dense(M)
    ev = np.linalg.eigvals(M).real
    _fd_check(A, 0.8 * ev.min(), 1.2 * ev.max(), 20, 4, 4, entries=[1, 5, 17, A.nnz - 3])


def test_grad_theta_matches_exact_trace_matern():
    """With k >= n the frozen estimator is the exact polynomial trace, so
    sum_e g_e da_e/dtheta = tr(p'(A) dA/dtheta) ~ tr(A^-1 dA/dtheta): n/tau for tau and
    4 kappa sum 1/(kappa^2 + mu) for kappa."""
    N, kappa, tau = 6, 0.3, 1.3
    A = matern_2d(N, kappa, tau)
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    lmin, lmax = 0.95 * lam[0], 1.05 * lam[-1]
    m = 200
    S, G = logdet.make_probes(A.n, A.n, seed=1)
    r = logdet.hutchpp_logdet(A, lmin, lmax, m, S, G)
    g = logdet.hutchpp_grad_values(A, lmin, lmax, m, r["Q"], r["Gp"])
    dk, dt = matern_2d_derivatives(N, kappa, tau)
    ex_k, ex_t = pins.dlogdet_matern_2d(N, kappa, tau)
    assert float(g @ dt) == pytest.approx(ex_t, rel=1e-5)
    assert float(g @ dk) == pytest.approx(ex_k, rel=1e-5)
    # the gradient of a symmetric matrix's estimator is symmetric
    Gm = __import__("scipy.sparse", fromlist=["csr_matrix"]).csr_matrix((g, A.colind, A.rowptr), shape=(A.n, A.n))
    assert abs(Gm - Gm.T).max() <= 1e-10 * abs(Gm).max()


@pytest.mark.parametrize("kappa,m", [(81.0, 39), (8080.0, 80), (2.5e6, 150), (1e9, 250)])
def test_divided_difference_table_vs_high_precision(kappa, m):
    """The xi-variable table (used when Algorithm 1's series is too long) against the 120-digit
    table in the z variable (Eq. Léja7)."""
    xi = leja.fast_leja_points(m + 1)
    c, g = (1.0 + kappa) / 2, (kappa - 1.0) / 4
    d = divdiff.divided_differences_table(xi, c, g)
    ref = pins.hp_scaled_divided_differences(1.0, kappa, xi)
    assert np.max(np.abs(d - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_divided_difference_method_choice():
    # config-3-like conditioning stays on Algorithm 1, config-5-like switches to the table
    _, _, _, d3, p3 = logdet.newton_leja_setup(1.0, 8080.0, 80)
    assert p3 > 0
    _, _, _, d5, p5 = logdet.newton_leja_setup(1.0, 2.5e6, 150)
    assert p5 == 0
    # s = lambda_max / 2 has q = 1: always the table, and the same coefficients as s = c
    _, _, _, dh, ph = logdet.newton_leja_setup(1.0, 50.0, 40, s_mode="half_lmax")
    _, _, _, dc, pc = logdet.newton_leja_setup(1.0, 50.0, 40)
    assert ph == 0 and pc > 0
    assert np.max(np.abs(dh - dc)) <= 1e-13 * np.max(np.abs(dc))


def test_banded_cholesky_pin_matches_dense():
    """The banded-Cholesky log-determinant used as ground truth for the pentadiagonal family
    agrees with NumPy's dense slogdet."""
    from synth import pentadiagonal
    A = pentadiagonal(300, seed=4)
    sign, ld = np.linalg.slogdet(A.to_scipy().toarray())
    assert sign == 1.0
    assert pins.logdet_banded(A) == pytest.approx(ld, rel=1e-13)


def test_hutchpp_pentadiagonal_exact_trace_against_banded_cholesky():
    """The paper's synthetic pentadiagonal family (Section 5.1). With as many sketch columns as
    rows the estimate is the exact polynomial trace, and on this spectrum (condition number
    about 1 + 16/n) the degree-10 interpolant is exact to rounding: the estimate equals the
    banded-Cholesky log-determinant."""
    from synth import pentadiagonal
    A = pentadiagonal(240, seed=7)
    lo, hi = logdet.gershgorin(A)
    sigma = logdet.sigma_of(lo)
    m = logdet.degree_from_bounds(lo / sigma, hi / sigma)
    S, G = logdet.make_probes(A.n, A.n, seed=3)
    r = logdet.hutchpp_logdet(A, lo, hi, m, S, G)
    assert r["estimate"] == pytest.approx(pins.logdet_banded(A), rel=1e-12)


def test_hutchpp_pentadiagonal_residual_variance():
    """With few probes the error on this family is Hutch++'s residual variance, not the
    interpolant: the large constant diagonal part n I is estimated exactly by Rademacher
    Hutchinson but not after the deflation (||(I - QQ^T) g||^2 varies). The error shrinks with
    the probe count and stays within a few standard deviations of log(n) sqrt(2)."""
    from synth import pentadiagonal
    A = pentadiagonal(2000, seed=4)
    lo, hi = logdet.gershgorin(A)
    m = logdet.degree_from_bounds(lo, hi)
    exact = pins.logdet_banded(A)
    errs = [abs(logdet.logdet_leja(A, lo, hi, m, probes, seed)["estimate"] - exact) for probes, seed in ((30, 1), (30, 2), (30, 3))]
    assert max(errs) < 6.0 * math.log(A.n) * math.sqrt(2.0)


def test_hutchinson_all_sign_vectors_is_the_exact_polynomial_trace():
    """Eq. Léja8: the mean of g^T F g over all 2^n sign vectors is tr F exactly (the cross terms
    cancel pairwise), so with every sign vector as a probe the estimate is n log sigma +
    sum_i p(lambda_i / sigma), computed here from a dense eigendecomposition."""
    import itertools
    A = random_spd(8, seed=3)
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    lmin, lmax = 0.9 * lam[0], 1.1 * lam[-1]
    G = np.array(list(itertools.product([-1.0, 1.0], repeat=A.n))).T   # 8 x 256
    r = logdet.hutchinson_logdet(A, lmin, lmax, 25, G)
    sigma = logdet.sigma_of(lmin)
    p = pins.interpolant(lmin / sigma, lmax / sigma, leja.fast_leja_points(26))
    assert r["estimate"] == pytest.approx(A.n * math.log(sigma) + float(np.sum(p(lam / sigma))), rel=1e-12)


def test_hutchinson_rademacher_exact_on_diagonal_matrices():
    """For a diagonal matrix every Rademacher probe gives g^T F g = tr F (g_i^2 = 1)."""
    dvals = np.linspace(0.3, 5.0, 57)
    A = diagonal(dvals)
    r = logdet.logdet_hutchinson(A, 0.3, 5.0, 30, 3, seed=9)
    sigma = logdet.sigma_of(0.3)
    p = pins.interpolant(0.3 / sigma, 5.0 / sigma, leja.fast_leja_points(31))
    assert r["estimate"] == pytest.approx(A.n * math.log(sigma) + float(np.sum(p(dvals / sigma))), rel=1e-12)


def test_hutchinson_uses_the_g_stream_columns():
    """The Hutchinson probes are the first columns of Algorithm 3's G stream."""
    A = laplacian_2d(10, 0.5)
    G = rng.probes("gaussian", 4, rng.STREAM_G, A.n, 6)
    a = logdet.hutchinson_logdet(A, 0.5, 8.5, 20, G)["estimate"]
    b = logdet.logdet_hutchinson(A, 0.5, 8.5, 20, 6, 4, kind="gaussian")["estimate"]
    assert a == b


# ------------------------------------------------------------------ Algorithm 2's stopping rule

def _first_at_or_below(e, tol):
    """Algorithm 2's loop: the first m with e_m <= tol, else the last index."""
    for m, em in enumerate(e):
        if not em > tol:
            return m
    return len(e) - 1


def _tol_stopping_at(e, lo):
    """A tolerance at which the rule stops at some m >= lo, with a wide margin on both sides:
    e_m below half of every earlier e_j, and tol their geometric mean."""
    for m in range(max(lo, 1), len(e)):
        prev = min(e[:m])
        if e[m] < 0.5 * prev:
            return m, math.sqrt(e[m] * prev)
    raise AssertionError("no clear stopping point")


def test_adaptive_degree_diagonal_closed_form():
    """Algorithm 2's stopping rule on a diagonal matrix, where w_m = prod_{j<m} (b_i - xi_j) v_i
    elementwise (b_i the scaled eigenvalues): the term norms |d_m| ||w_m|| come from these
    products and 120-digit divided differences, the result from the barycentric interpolant of
    the stopping degree. Columns of different scale stop at different degrees."""
    n, lmin, lmax, mmax = 64, 0.3, 7.0, 60
    lam = np.linspace(lmin, lmax, n)
    A = diagonal(lam)
    sigma = logdet.sigma_of(lmin)
    lt, ut = lmin / sigma, lmax / sigma
    xi = leja.fast_leja_points(mmax + 1)
    c, g = (lt + ut) / 2, (ut - lt) / 4
    dh = pins.hp_scaled_divided_differences(lt, ut, xi)
    b = (lam / sigma - c) / g
    omega = np.concatenate([np.ones((n, 1)), np.cumprod(b[:, None] - xi[None, :mmax], axis=1)], axis=1)
    v0 = rng.rademacher(5, 0, n, 1)[:, 0]
    scales = [1.0, 1e-3, 1e3]
    V = np.stack([s * v0 for s in scales], axis=1)
    e0 = np.abs(dh) * np.sqrt(np.sum((omega * v0[:, None]) ** 2, axis=0))
    m0, tol = _tol_stopping_at(e0, 12)
    want = [_first_at_or_below(s * e0, tol) for s in scales]
    assert want[1] < want[0] < want[2]
    xi_o, c_o, g_o, d_o, _ = logdet.newton_leja_setup(lt, ut, mmax)
    P, deg = logdet.leja_apply_columns_adaptive(logdet._scipy(A), V, xi_o, d_o, c_o, g_o, tol, sigma)
    assert deg.tolist() == want
    for col, m in enumerate(want):
        p = pins.interpolant(lt, ut, xi[: m + 1])
        ref = p(lam / sigma) * V[:, col]
        assert np.max(np.abs(P[:, col] - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_adaptive_degree_dense_brute_force():
    """On a small dense SPD matrix the Newton basis is formed as explicit matrix products
    prod_{j<m} (B - xi_j I), B = (A / sigma - c I) / gamma, and applied to each column; the
    stopping degrees and the truncated sums match the recurrence of the oracle."""
    A = random_spd(7, seed=11)
    Ad = A.to_scipy().toarray()
    lam = np.linalg.eigvalsh(Ad)
    lmin, lmax, mmax = 0.8 * lam[0], 1.2 * lam[-1], 40
    sigma = logdet.sigma_of(lmin)
    xi, c, g, d, _ = logdet.newton_leja_setup(lmin / sigma, lmax / sigma, mmax)
    B = (Ad / sigma - c * np.eye(A.n)) / g
    mats = [np.eye(A.n)]
    for j in range(mmax):
        mats.append((B - xi[j] * np.eye(A.n)) @ mats[-1])
    V = np.random.default_rng(2).standard_normal((A.n, 3)) * np.array([1.0, 50.0, 0.02])
    e = np.array([[abs(d[m]) * np.linalg.norm(mats[m] @ V[:, col]) for m in range(mmax + 1)] for col in range(3)])
    _, tol = _tol_stopping_at(e[0], 8)
    want = [_first_at_or_below(e[col], tol) for col in range(3)]
    P, deg = logdet.leja_apply_columns_adaptive(logdet._scipy(A), V, xi, d, c, g, tol, sigma)
    assert deg.tolist() == want
    for col, m in enumerate(want):
        ref = sum(d[j] * (mats[j] @ V[:, col]) for j in range(m + 1))
        assert np.max(np.abs(P[:, col] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_adaptive_degree_tiny_tol_is_the_fixed_degree():
    """A tolerance below every term norm runs every column to the cap, with the fixed-degree
    arithmetic unchanged."""
    A = laplacian_2d(9, 0.4)
    V = rng.rademacher(2, 0, A.n, 3)
    xi, c, g, d, _ = logdet.newton_leja_setup(0.4, 8.4, 30)
    M = logdet._scipy(A)
    P, deg = logdet.leja_apply_columns_adaptive(M, V, xi, d, c, g, 1e-300)
    assert deg.tolist() == [30, 30, 30]
    assert np.array_equal(P, logdet.leja_apply_columns(M, V, xi, d, c, g))
    with pytest.raises(ValueError):
        logdet.leja_apply_columns_adaptive(M, V, xi, d, c, g, 0.0)


def test_adaptive_hutchinson_diagonal_closed_form():
    """Rademacher probes on a diagonal matrix: every column has the same term norms
    |d_m| sqrt(sum_i omega_m(b_i)^2), so every column stops at the same degree, and the
    estimate is n log sigma + sum_i p(lambda_i / sigma) with p the interpolant of that degree."""
    n, lmin, lmax, mmax = 80, 0.2, 6.0, 70
    lam = np.linspace(lmin, lmax, n) ** 1.0
    A = diagonal(lam)
    sigma = logdet.sigma_of(lmin)
    lt, ut = lmin / sigma, lmax / sigma
    xi = leja.fast_leja_points(mmax + 1)
    c, g = (lt + ut) / 2, (ut - lt) / 4
    dh = pins.hp_scaled_divided_differences(lt, ut, xi)
    b = (lam / sigma - c) / g
    omega = np.concatenate([np.ones((n, 1)), np.cumprod(b[:, None] - xi[None, :mmax], axis=1)], axis=1)
    e = np.abs(dh) * np.sqrt(np.sum(omega ** 2, axis=0))
    m, tol = _tol_stopping_at(e, 15)
    r = logdet.logdet_hutchinson(A, lmin, lmax, mmax, 4, seed=3, tol=tol)
    assert r["deg_g"].tolist() == [m] * 4
    p = pins.interpolant(lt, ut, xi[: m + 1])
    assert r["estimate"] == pytest.approx(n * math.log(sigma) + float(np.sum(p(lam / sigma))), rel=1e-12)


def test_adaptive_hutchpp_degrees_and_accuracy_follow_tol():
    """Hutch++ with the rule in both passes: a smaller tolerance never stops a column earlier,
    the estimate approaches the fixed-degree estimate at the cap, and at a tolerance below
    every term it equals it."""
    A = laplacian_2d(16, 0.2)
    lo, hi = 0.2, 8.2
    fixed = logdet.logdet_leja(A, lo, hi, 80, 12, seed=4)["estimate"]
    prev, errs = None, []
    for tol in (1e-1, 1e-3, 1e-5, 1e-7):
        r = logdet.logdet_leja(A, lo, hi, 80, 12, seed=4, tol=tol)
        degs = np.concatenate([r["deg_s"], r["deg_q"], r["deg_g"]])
        assert degs.min() >= 1 and degs.max() <= 80
        if prev is not None:
            assert np.all(degs >= prev)
        prev = degs
        errs.append(abs(r["estimate"] - fixed))
    assert errs[0] > errs[1] > errs[2] > errs[3]
    r = logdet.logdet_leja(A, lo, hi, 80, 12, seed=4, tol=1e-300)
    assert r["estimate"] == fixed


# ------------------------------------------------ the GMRF of the maximum-likelihood experiment

@pytest.mark.parametrize("theta", [-0.24, -0.22, -0.1, 0.2])
def test_gmrf_theta_closed_form_vs_dense(theta):
    """Q(theta) = I + theta Adj on a 9 x 9 grid: the closed-form log-determinant and its
    theta-derivative (Section 5.3's model) against a dense LU and tr(Q^-1 Adj)."""
    from synth import gmrf_theta
    N = 9
    Q = gmrf_theta(N, theta).to_scipy().toarray()
    Adj = Q - np.eye(N * N)
    Adj = Adj / theta
    sign, ld = np.linalg.slogdet(Q)
    assert sign > 0
    assert pins.logdet_gmrf_theta(N, theta) == pytest.approx(ld, rel=1e-13)
    assert pins.dlogdet_gmrf_theta(N, theta) == pytest.approx(np.trace(np.linalg.solve(Q, Adj)), rel=1e-11)


def test_gmrf_theta_bounds_and_sigma():
    """Gershgorin gives the paper's interval [1 - 4|theta|, 1 + 4|theta|] (interior rows have four
    neighbours), so sigma = 1 - 4|theta| as Section 5.3 sets it."""
    from synth import gmrf_theta
    for theta in (-0.22, 0.15):
        lo, hi = logdet.gershgorin(gmrf_theta(12, theta))
        assert lo == pytest.approx(1 - 4 * abs(theta), abs=1e-15)
        assert hi == pytest.approx(1 + 4 * abs(theta), abs=1e-15)
        assert logdet.sigma_of(lo) == pytest.approx(1 - 4 * abs(theta), abs=1e-15)


def test_gmrf_theta_exact_trace_against_closed_form():
    """With k >= n the Hutch++ estimate is the exact polynomial trace n log sigma + tr p(Q~);
    at degree 70 on kappa <= 49 it matches the closed-form log-determinant to 1e-9."""
    from synth import gmrf_theta
    N, theta = 7, -0.24
    A = gmrf_theta(N, theta)
    lo, hi = logdet.gershgorin(A)
    r = logdet.logdet_leja(A, lo, hi, 70, 3 * A.n, seed=2)
    assert r["estimate"] == pytest.approx(pins.logdet_gmrf_theta(N, theta), rel=1e-9, abs=1e-9)


# ------------------------------------------------------ derivative through the sketch's QR

def _estimate_with_values(A, values, lmin, lmax, degree, S, G):
    from synth import CSR
    B = CSR(A.n, A.rowptr, A.colind, np.asarray(values, dtype=np.float64))
    return logdet.hutchpp_logdet(B, lmin, lmax, degree, S, G)["estimate"]


@pytest.mark.parametrize("seed", [0, 1])
def test_full_gradient_matches_finite_differences(seed):
    """Central differences of Algorithm 3's estimate (S, G, bounds and degree fixed; Q and G'
    recomputed from the perturbed matrix by Householder QR) against the frozen-basis gradient
    plus the term through the QR. The QR term is far above the differencing error, so dropping
    it, or a wrong sign or factor in it, fails."""
    A = random_spd(40, nnz_per_row=5, seed=seed)
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    lmin, lmax, degree = 0.9 * lam[0], 1.1 * lam[-1], 18
    S = rng.rademacher(seed, rng.STREAM_S, A.n, 4)
    G = rng.rademacher(seed, rng.STREAM_G, A.n, 4)
    full = logdet.hutchpp_full_grad_values(A, lmin, lmax, degree, S, G)
    r = logdet.hutchpp_logdet(A, lmin, lmax, degree, S, G)
    frozen = logdet.hutchpp_grad_values(A, lmin, lmax, degree, r["Q"], r["Gp"])
    picks = np.random.default_rng(seed).choice(A.nnz, 14, replace=False)
    for e in picks:
        h = 1e-5 * max(1.0, abs(A.values[e]))
        vp, vm = A.values.copy(), A.values.copy()
        vp[e] += h
        vm[e] -= h
        fd = (_estimate_with_values(A, vp, lmin, lmax, degree, S, G) -
              _estimate_with_values(A, vm, lmin, lmax, degree, S, G)) / (2 * h)
        assert full[e] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    assert np.max(np.abs(full - frozen)) > 1e3 * 1e-6 * np.max(np.abs(full))


def test_full_gradient_equals_frozen_when_the_sketch_spans_everything():
    """k = n: span(Y) = R^n, Pi = I, G' = 0 and Gamma = 2 (I - Pi) Z Q R^-T = 0."""
    A = random_spd(9, seed=2)
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    S = rng.gaussian(1, rng.STREAM_S, A.n, A.n)
    G = rng.gaussian(1, rng.STREAM_G, A.n, A.n)
    w = logdet.hutchpp_qr_weights(A, 0.9 * lam[0], 1.1 * lam[-1], 20, S, G)
    assert np.max(np.abs(w["Gamma"])) < 1e-10 * np.max(np.abs(w["FQ"]))
