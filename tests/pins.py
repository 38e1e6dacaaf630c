"""Independent references that pin the oracle (and, through it, the CUDA path).

None of these routines calls the oracle. They restate the mathematics by another route:
  * divided differences by the textbook recurrence (Section 3.1, Eq. Léja7) in 120-digit
    decimal arithmetic;
  * the interpolating polynomial by SciPy's barycentric Lagrange interpolation;
  * matrix functions by a dense symmetric eigendecomposition;
  * log-determinants of shifted Laplacians and Matérn operators in closed form;
  * log-determinants of banded SPD matrices by LAPACK's banded Cholesky (SciPy).
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext

import numpy as np
from scipy.interpolate import BarycentricInterpolator


def hp_scaled_divided_differences(lmin: float, lmax: float, xi, prec: int = 120, c_g=None) -> np.ndarray:
    """gamma^j * log[z_0, ..., z_j] with z_i = c + gamma xi_i, c = (lmin+lmax)/2,
    gamma = (lmax-lmin)/4, by the standard divided-difference table in `prec` digits. c_g = (c,
    gamma) given as floats puts the nodes where an implementation that rounds c and gamma to
    FP64 puts them."""
    getcontext().prec = prec
    lo, hi = Decimal(lmin), Decimal(lmax)
    c = (lo + hi) / 2
    g = (hi - lo) / 4
    if c_g is not None:
        c, g = Decimal(c_g[0]), Decimal(c_g[1])
    z = [c + g * Decimal(float(x)) for x in xi]
    m1 = len(z)
    col = [zi.ln() for zi in z]            # f[z_i]
    coef = [col[0]]
    for order in range(1, m1):
        col = [(col[i + 1] - col[i]) / (z[i + order] - z[i]) for i in range(m1 - order)]
        coef.append(col[0])                # f[z_0, ..., z_order]
    return np.array([float(coef[j] * g ** j) for j in range(m1)])


def newton_value_hp(d, xi, lmin: float, lmax: float, x: float, prec: int = 60) -> float:
    """Evaluate sum_j d_j prod_{k<j} ((x - c)/gamma - xi_k) in high precision."""
    getcontext().prec = prec
    lo, hi = Decimal(lmin), Decimal(lmax)
    c = (lo + hi) / 2
    g = (hi - lo) / 4
    t = (Decimal(x) - c) / g
    acc = Decimal(0)
    basis = Decimal(1)
    for j in range(len(d)):
        acc += Decimal(float(d[j])) * basis
        basis *= t - Decimal(float(xi[j]))
    return float(acc)


def interpolant(lmin: float, lmax: float, xi):
    """The polynomial interpolating log at z_i = c + gamma xi_i, as a callable (barycentric)."""
    c = (lmin + lmax) / 2.0
    g = (lmax - lmin) / 4.0
    xi = np.asarray(xi, dtype=np.float64)
    bary = BarycentricInterpolator(xi, np.log(c + g * xi))
    return lambda x: bary((np.asarray(x, dtype=np.float64) - c) / g)


def dense_matrix_function(Adense: np.ndarray, f) -> np.ndarray:
    lam, U = np.linalg.eigh(Adense)
    return (U * f(lam)) @ U.T


def lap_eigs_1d(N: int) -> np.ndarray:
    i = np.arange(1, N + 1)
    return 4.0 * np.sin(i * np.pi / (2.0 * (N + 1))) ** 2


def logdet_laplacian_2d(N: int, shift: float) -> float:
    mu = lap_eigs_1d(N)
    return math.fsum(np.log(mu[:, None] + mu[None, :] + shift).ravel())


def logdet_laplacian_3d(N: int, shift: float) -> float:
    mu = lap_eigs_1d(N)
    s2 = (mu[:, None] + mu[None, :]).ravel()
    return math.fsum(math.fsum(np.log(s2 + m + shift)) for m in mu)


def logdet_matern_2d(N: int, kappa: float, tau: float) -> float:
    mu = lap_eigs_1d(N)
    s2 = (mu[:, None] + mu[None, :]).ravel()
    return N * N * math.log(tau) + 2.0 * math.fsum(np.log(kappa * kappa + s2))


def dlogdet_matern_2d(N: int, kappa: float, tau: float) -> tuple[float, float]:
    """(d/dkappa, d/dtau) of log det tau (kappa^2 I + L)^2: 4 kappa sum 1/(kappa^2 + mu), n / tau."""
    mu = lap_eigs_1d(N)
    s2 = (mu[:, None] + mu[None, :]).ravel()
    return 4.0 * kappa * math.fsum(1.0 / (kappa * kappa + s2)), N * N / tau


def adj_eigs_1d(N: int) -> np.ndarray:
    """Eigenvalues of the path graph's adjacency: 2 cos(i pi / (N + 1)), i = 1..N."""
    return 2.0 * np.cos(np.arange(1, N + 1) * np.pi / (N + 1))


def logdet_gmrf_theta(N: int, theta: float) -> float:
    """log det (I + theta Adj) on the N x N grid: sum_ij log(1 + theta (a_i + a_j))."""
    a = adj_eigs_1d(N)
    return math.fsum(math.fsum(np.log1p(theta * (a + ai))) for ai in a)


def dlogdet_gmrf_theta(N: int, theta: float) -> float:
    """d/dtheta log det (I + theta Adj) = sum_ij (a_i + a_j) / (1 + theta (a_i + a_j))."""
    a = adj_eigs_1d(N)
    return math.fsum(math.fsum((a + ai) / (1.0 + theta * (a + ai))) for ai in a)


def logdet_banded(A, bandwidth: int = 2) -> float:
    """log det A = 2 sum_i log(R_ii) for a symmetric positive definite CSR matrix whose entries lie
    within `bandwidth` of the diagonal, from LAPACK's banded Cholesky (SciPy) in O(n)."""
    from scipy.linalg import cholesky_banded
    M = A.to_scipy() if hasattr(A, "to_scipy") else A
    M = M.tocsr()
    n = M.shape[0]
    ab = np.zeros((bandwidth + 1, n))
    for k in range(bandwidth + 1):   # upper form: ab[bandwidth - k, j] = A[j - k, j]
        ab[bandwidth - k, k:] = M.diagonal(k)
    R = cholesky_banded(ab, lower=False)
    return 2.0 * math.fsum(np.log(R[bandwidth]))
