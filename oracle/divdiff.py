"""Divided differences of log at mapped Léja points via Algorithm 1 (oracle; test infrastructure only).

Section 3.1, Algorithm 1: with nodes z_i = c + gamma * xi_i (Eq. z_mapping), the Léja matrix
Qhat_m is lower bidiagonal with diagonal xi_0..xi_m and ones below it (Eq. eq_leja_matrix),
Q_m = c I + gamma Qhat_m, W_m = (Q_m - s I) / s, and

    d = log(Q_m) e_1 = (log(s) I + log(I + W_m)) e_1,

with log(I + W_m) a Taylor series sum_{k>=1} (-1)^{k+1} W_m^k / k.

Because Q_m = D Z D^{-1} with D = diag(gamma^j) and Z lower bidiagonal with diagonal z and unit
sub-diagonal, the first column of log(Q_m) is (gamma^j * log[z_0, ..., z_j])_j: the scaled
Newton coefficients d_j used by the scaled recurrence in logdet.py.

Readings fixed by this library (the paper is silent or inconsistent):
  * gamma = (lambda_max - lambda_min) / 4 as in Eq. eq_gamma (Algorithms 1 and 2 print /2, which
    would map [-2, 2] outside the spectral interval);
  * Q_m = c I + gamma Qhat_m as in Algorithm 1 step 5 (the text before it prints a minus sign);
  * the Taylor order is adaptive: terms are added until the max-norm of a term is below
    1e-18 times the max-norm of the running sum, after at least 10 terms; more than
    5,000,000 terms raises DividedDifferenceError;
  * s defaults to c, the optimum of Lemma 3.1; s = lambda_max / 2 is the other choice the paper
    reports;
  * when the series would need more than 1e6 terms (predicted from its convergence factor
    q = max_i |z_i / s - 1|, i.e. ln(1e-18) / ln(q) > 1e6, which happens for condition numbers
    above ~1e5 at s = c and always at s = lambda_max / 2), the divided differences are taken
    from the textbook table (Eq. Léja7) of g(xi) = log(c + gamma xi) over the Léja points on
    [-2, 2] instead: since z = c + gamma xi, g[xi_0..xi_j] = gamma^j log[z_0..z_j] = d_j exactly,
    and in this variable the table neither underflows nor loses accuracy for Léja-ordered nodes.
"""
from __future__ import annotations

import math

import numpy as np

TAYLOR_REL_TOL = 1e-18
TAYLOR_MIN_TERMS = 10
TAYLOR_MAX_TERMS = 5_000_000


class DividedDifferenceError(RuntimeError):
    pass


TABLE_THRESHOLD_TERMS = 1_000_000


def predicted_taylor_terms(xi: np.ndarray, c: float, gamma: float, s: float) -> float:
    """ln(1e-18) / ln(q) with q = max_i |z_i / s - 1| (infinite when q >= 1)."""
    q = float(np.max(np.abs((c + gamma * np.asarray(xi, dtype=np.float64)) / s - 1.0)))
    if q >= 1.0:
        return math.inf
    if q <= 0.0:
        return 1.0
    return math.log(TAYLOR_REL_TOL) / math.log(q)


def divided_differences_table(xi: np.ndarray, c: float, gamma: float) -> np.ndarray:
    """d_j = g[xi_0, ..., xi_j] for g(xi) = log(c + gamma xi) by the standard recurrence
    (Eq. Léja7) in the xi variable: column o holds g[xi_i, ..., xi_{i+o}]."""
    xi = np.asarray(xi, dtype=np.float64)
    col = np.log(c + gamma * xi)
    out = [col[0]]
    for o in range(1, xi.shape[0]):
        col = (col[1:] - col[:-1]) / (xi[o:] - xi[:-o])
        out.append(col[0])
    return np.array(out)


def scaled_divided_differences(xi: np.ndarray, c: float, gamma: float, s: float | None = None) -> tuple[np.ndarray, int]:
    """Algorithm 1 when its series converges in a reasonable number of terms, otherwise the
    xi-variable table. Returns (d, p) with p = 0 when the table was used."""
    if s is None:
        s = c
    if predicted_taylor_terms(xi, c, gamma, s) > TABLE_THRESHOLD_TERMS:
        return divided_differences_table(xi, c, gamma), 0
    return divided_differences(xi, c, gamma, s)


def divided_differences(xi: np.ndarray, c: float, gamma: float, s: float | None = None,
                        max_terms: int = TAYLOR_MAX_TERMS) -> tuple[np.ndarray, int]:
    """Algorithm 1: d = log(Q_m) e_1 for the nodes z_i = c + gamma * xi_i.

    Returns (d, p) with p the number of Taylor terms used.
    """
    xi = np.asarray(xi, dtype=np.float64)
    m1 = xi.shape[0]
    if s is None:
        s = c
    if not (s > 0.0):
        raise ValueError("s_val must be positive")
    # steps 4-6: Q_m = c I + gamma Qhat_m and W_m = (Q_m - s I) / s, both lower bidiagonal
    qm_diag = c + gamma * xi
    qm_sub = gamma
    w_diag = (qm_diag - s) / s
    w_sub = qm_sub / s
    # step 7: log(I + W_m) e_1 by the Taylor series, applying W_m to a vector each term
    t = np.zeros(m1)
    t[0] = 1.0
    acc = np.zeros(m1)
    p = 0
    for k in range(1, max_terms + 1):
        t_new = w_diag * t
        t_new[1:] += w_sub * t[:-1]
        t = t_new
        term = t / k if k % 2 == 1 else -t / k
        acc = acc + term
        p = k
        if k >= TAYLOR_MIN_TERMS and np.max(np.abs(term)) < TAYLOR_REL_TOL * np.max(np.abs(acc)):
            break
    else:
        raise DividedDifferenceError(f"Taylor series not converged after {max_terms} terms")
    # step 8: log(Q_m) e_1 = log(s) e_1 + log(I + W_m) e_1
    d = acc.copy()
    d[0] += math.log(s)
    return d, p
