"""Léja-point log-determinant estimator, step by step in FP64 (oracle; test infrastructure only).

Follows arXiv 2603.02207:
  * spectral bounds by Gershgorin's theorem (Section 3; Algorithm 1 step 1; Remark on
    non-positive lower bounds), with an optional power-iteration refinement of lambda_max in
    the spirit of the Lanczos alternative (Appendix A);
  * sigma-normalisation Q~ = Q / sigma when lambda_min < 1 (Section 4, Eq. scaled_sigma_matrix)
    and log det Q = n log sigma + tr log Q~;
  * Algorithm 2 (Newton-Léja action p(Q~)v), applied column by column, to a fixed degree or
    with its stopping rule |d_m| ||w_m||_2 <= tol;
  * Hutch++ as in Algorithm 3 / Section 4.1 (sketch, Householder QR, deterministic part,
    Hutchinson part on the deflated probes);
  * the plain Hutchinson estimator the paper starts from (Eq. Léja8), on the same probes;
  * the derivative of the frozen-basis estimator with respect to the stored matrix values, and
    the derivative through the sketch's QR (Algorithm 3 step 4).

Readings fixed by this library where the paper is silent or ambiguous:
  * the operator in Algorithm 2's update (Q - xi_m I) is the scaled operator
    B = (Q~ - c I) / gamma with xi_m in [-2, 2]; with d_j = gamma^j log[z_0..z_j] from
    Algorithm 1 this equals the unscaled Newton form at z_j = c + gamma xi_j exactly in exact
    arithmetic, and keeps the Newton basis O(1);
  * "degree m" means m+1 Léja points, coefficients d_0..d_m and m operator applications;
  * Algorithm 2 runs either to a fixed degree (tol = 0) or with its stopping rule (tol > 0):
    column by column, the loop stops at the first m with |d_m| ||w_m||_2 <= tol, and the term
    d_m w_m that met the rule is kept (P_m already holds it when the test is made); the number
    of Léja points caps m at the degree given; in Hutch++ both the sketch pass and the trace
    pass use the rule, each column on its own;
  * a non-positive lower bound is an error (the caller supplies a positive one);
  * sigma = lambda_min when lambda_min < 1, else 1;
  * the residual normalisation of Eq. eq_lej_residual_def is 1/k with k = m_vec / 3;
  * the QR of step 4 is Householder (NumPy/LAPACK); any orthonormal basis of span(Y) gives the
    same estimate;
  * the gradient differentiates the estimator with Q, the deflated probes, the bounds, sigma
    and the coefficients d held fixed, per stored CSR entry; the full gradient also carries the
    derivative through Q = orth(p(A~) S) and G' (the bounds, sigma and d still fixed);
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from .divdiff import scaled_divided_differences
from .leja import fast_leja_points
from . import rng as _rng


def _scipy(A) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(A.values, dtype=np.float64), A.colind, A.rowptr), shape=(A.n, A.n))


# ---------------------------------------------------------------------------------------------
# bounds and normalisation
# ---------------------------------------------------------------------------------------------

def gershgorin(A) -> tuple[float, float]:
    """Gershgorin interval [min_i (a_ii - R_i), max_i (a_ii + R_i)], R_i = sum_{j != i} |a_ij|,
    row by row in ascending column order (Section 3; Algorithm 1 step 1)."""
    if A.n == 0:
        return 0.0, 0.0
    vals = np.asarray(A.values, dtype=np.float64)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    is_diag = np.asarray(A.colind) == rows
    a_ii = np.zeros(A.n)
    r_i = np.zeros(A.n)
    # np.add.at accumulates unbuffered in index order: ascending column within each row
    np.add.at(a_ii, rows[is_diag], vals[is_diag])
    np.add.at(r_i, rows[~is_diag], np.abs(vals[~is_diag]))
    return float(np.min(a_ii - r_i)), float(np.max(a_ii + r_i))


def power_iteration_lmax(A, iters: int = 20, seed: int = 0) -> float:
    """Rayleigh quotient after `iters` normalised power steps from the stream-2 Rademacher
    vector (a cheap stand-in for the Lanczos lambda_max of Appendix A)."""
    M = _scipy(A)
    v = _rng.rademacher(seed, _rng.STREAM_POWER, A.n, 1)[:, 0]
    v = v / np.linalg.norm(v)
    for _ in range(iters):
        w = M @ v
        v = w / np.linalg.norm(w)
    return float(v @ (M @ v))


def sigma_of(lmin: float) -> float:
    """Section 4, Eq. scaled_sigma_matrix: sigma = lambda_min if lambda_min < 1, else 1."""
    if not (lmin > 0.0):
        raise ValueError("lower spectral bound must be positive")
    return lmin if lmin < 1.0 else 1.0


def degree_from_bounds(lmin: float, lmax: float, target: float = 1e-6, lo: int = 10, hi: int = 250) -> int:
    """Degree from the convergence rate of Proposition 3.1: rho = (sqrt(k)+1)/(sqrt(k)-1),
    m = ceil(ln(1/target) / ln(rho)), clamped to [lo, hi]."""
    kappa = lmax / lmin
    sk = math.sqrt(kappa)
    rho = (sk + 1.0) / (sk - 1.0)
    m = math.ceil(math.log(1.0 / target) / math.log(rho))
    return max(lo, min(hi, m))


# ---------------------------------------------------------------------------------------------
# Newton-Léja interpolant of log
# ---------------------------------------------------------------------------------------------

def newton_leja_setup(lmin: float, lmax: float, degree: int, s_mode: str = "center"):
    """Léja points on [-2, 2], the map z = c + gamma xi (Eqs. z_mapping, eq_centre, eq_gamma)
    and the scaled coefficients d_0..d_degree by Algorithm 1 (or the xi-variable divided
    difference table when Algorithm 1's series would need more than 1e6 terms; p = 0 then)."""
    if not (0.0 < lmin < lmax):
        raise ValueError("need 0 < lmin < lmax")
    xi = fast_leja_points(degree + 1)
    c = (lmin + lmax) / 2.0
    gamma = (lmax - lmin) / 4.0
    if s_mode == "center":
        s = c
    elif s_mode == "half_lmax":
        s = lmax / 2.0
    else:
        raise ValueError(s_mode)
    d, p = scaled_divided_differences(xi, c, gamma, s)
    return xi, c, gamma, d, p


def _round32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def leja_apply_columns(M: sp.csr_matrix, V: np.ndarray, xi, d, c: float, gamma: float,
                       scale: float = 1.0, f32: bool = False) -> np.ndarray:
    """Algorithm 2 with a fixed degree m = len(d) - 1, one column at a time:
    w_0 = v, P_0 = d_0 w_0; w_{j+1} = (B - xi_j I) w_j with B w = ((M w)/scale - c w)/gamma;
    P_{j+1} = P_j + d_{j+1} w_{j+1}.

    f32=True mirrors FP32 storage of the matrix values and of every w_j (the sums stay FP64).
    """
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    if f32:
        M = sp.csr_matrix((_round32(M.data), M.indices, M.indptr), shape=M.shape)
    m = len(d) - 1
    out = np.empty_like(V)
    for col in range(V.shape[1]):
        w = V[:, col].copy()
        if f32:
            w = _round32(w)
        P = d[0] * w
        for j in range(m):
            Bw = ((M @ w) / scale - c * w) / gamma
            w = Bw - xi[j] * w
            if f32:
                w = _round32(w)
            P = P + d[j + 1] * w
        out[:, col] = P
    return out


def leja_apply_columns_adaptive(M: sp.csr_matrix, V: np.ndarray, xi, d, c: float, gamma: float, tol: float,
                                scale: float = 1.0, f32: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Algorithm 2 with its stopping rule, one column at a time: w_0 = v, P_0 = d_0 w_0, m = 0;
    while |d_m| ||w_m||_2 > tol and m < len(d) - 1: w_{m+1} = (B - xi_m I) w_m, m = m + 1,
    P_m = P_{m-1} + d_m w_m. Returns (P for every column, the final m of every column).

    f32=True mirrors FP32 storage of the matrix values and of every w_j, as in
    leja_apply_columns; the norms are taken in FP64 of the stored w_j.
    """
    if not (tol > 0.0):
        raise ValueError("tol must be positive")
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 1:
        V = V[:, None]
    if f32:
        M = sp.csr_matrix((_round32(M.data), M.indices, M.indptr), shape=M.shape)
    mmax = len(d) - 1
    out = np.empty_like(V)
    degrees = np.zeros(V.shape[1], dtype=np.int64)
    for col in range(V.shape[1]):
        w = V[:, col].copy()
        if f32:
            w = _round32(w)
        P = d[0] * w
        m = 0
        while m < mmax and abs(d[m]) * np.linalg.norm(w) > tol:
            Bw = ((M @ w) / scale - c * w) / gamma
            w = Bw - xi[m] * w
            if f32:
                w = _round32(w)
            m += 1
            P = P + d[m] * w
        out[:, col] = P
        degrees[col] = m
    return out, degrees


def apply_poly(A, V: np.ndarray, lmin: float, lmax: float, degree: int, f32: bool = False,
               s_mode: str = "center") -> np.ndarray:
    """p_m(A) V, with p_m the degree-m Newton-Léja interpolant of log on [lmin, lmax]."""
    xi, c, gamma, d, _ = newton_leja_setup(lmin, lmax, degree, s_mode)
    return leja_apply_columns(_scipy(A), V, xi, d, c, gamma, 1.0, f32)


# ---------------------------------------------------------------------------------------------
# Hutch++ (Algorithm 3)
# ---------------------------------------------------------------------------------------------

def make_probes(n: int, k: int, seed: int, kind: str = "rademacher") -> tuple[np.ndarray, np.ndarray]:
    """Algorithm 3 steps 2 and 6: S (stream 0) and G (stream 1), each n x k."""
    return _rng.probes(kind, seed, _rng.STREAM_S, n, k), _rng.probes(kind, seed, _rng.STREAM_G, n, k)


def hutchpp_logdet(A, lmin: float, lmax: float, degree: int, S: np.ndarray, G: np.ndarray,
                   s_mode: str = "center", f32: bool = False, tol: float = 0.0) -> dict:
    """Algorithm 3: log det A ~ n log sigma + tr(Q^T F Q) + (1/k) sum_j g'_j^T F g'_j, with
    F = p(A / sigma), Q = orth(F S) and g'_j = (I - Q Q^T) g_j. With tol > 0 every application
    of F stops column by column by Algorithm 2's rule (degree is then the cap); the result holds
    the final degrees of the sketch pass (deg_s) and of the trace pass (deg_q, deg_g)."""
    n = A.n
    k = S.shape[1]
    sigma = sigma_of(lmin)
    # step 1: A~ = A / sigma, whose spectrum lies in [lmin / sigma, lmax / sigma]
    lt, ut = lmin / sigma, lmax / sigma
    xi, c, gamma, d, p_terms = newton_leja_setup(lt, ut, degree, s_mode)
    M = _scipy(A)
    degs = []

    def F(X):
        if tol > 0.0:
            out, dg = leja_apply_columns_adaptive(M, X, xi, d, c, gamma, tol, sigma, f32)
            degs.append(dg)
            return out
        return leja_apply_columns(M, X, xi, d, c, gamma, sigma, f32)

    # step 3: Y = F S
    Y = F(S)
    # step 4: orthonormal basis of span(Y) by Householder QR
    Q, _ = np.linalg.qr(Y, mode="reduced")
    # step 5: tr(Q^T F Q)
    Qin = _round32(Q) if f32 else Q
    FQ = F(Qin)
    t_q = float(np.sum(Qin * FQ))
    # step 6: deflated probes and the Hutchinson part
    Gp = G - Q @ (Q.T @ G)
    Gin = _round32(Gp) if f32 else Gp
    FG = F(Gin)
    kk = G.shape[1]
    t_r = float(np.sum(Gin * FG)) / kk if kk > 0 else 0.0
    # step 7 and output
    est = n * math.log(sigma) + t_q + t_r
    out = dict(estimate=est, trace_q=t_q, trace_res=t_r, sigma=sigma, c=c, gamma=gamma, xi=xi, d=d,
               taylor_terms=p_terms, Y=Y, Q=Q, Gp=Gp, k=k)
    if tol > 0.0:
        out.update(deg_s=degs[0], deg_q=degs[1], deg_g=degs[2])
    return out


def logdet_leja(A, lmin: float, lmax: float, degree: int, probes: int, seed: int,
                kind: str = "rademacher", s_mode: str = "center", f32: bool = False, tol: float = 0.0) -> dict:
    """logdet_leja(csr, bounds, degree, probes, seed): Algorithm 3 with probes = m_vec
    (a multiple of 3; k = m_vec / 3 columns each for S and G)."""
    if probes % 3 != 0 or probes <= 0:
        raise ValueError("probes must be a positive multiple of 3")
    k = probes // 3
    S, G = make_probes(A.n, k, seed, kind)
    return hutchpp_logdet(A, lmin, lmax, degree, S, G, s_mode, f32, tol)


# ---------------------------------------------------------------------------------------------
# plain Hutchinson (Eq. Léja8)
# ---------------------------------------------------------------------------------------------

def hutchinson_logdet(A, lmin: float, lmax: float, degree: int, G: np.ndarray, s_mode: str = "center",
                      f32: bool = False, tol: float = 0.0) -> dict:
    """Eq. Léja8 with the sigma-normalisation: log det A ~ n log sigma + (1/m) sum_j g_j^T F g_j
    over the m columns g_j of G, F = p(A / sigma); with tol > 0, F stops column by column by
    Algorithm 2's rule (the final degrees are returned as deg_g)."""
    n = A.n
    m = G.shape[1]
    sigma = sigma_of(lmin)
    lt, ut = lmin / sigma, lmax / sigma
    xi, c, gamma, d, p_terms = newton_leja_setup(lt, ut, degree, s_mode)
    Gin = _round32(G) if f32 else G
    dg = None
    if tol > 0.0:
        FG, dg = leja_apply_columns_adaptive(_scipy(A), Gin, xi, d, c, gamma, tol, sigma, f32)
    else:
        FG = leja_apply_columns(_scipy(A), Gin, xi, d, c, gamma, sigma, f32)
    t = float(np.sum(Gin * FG)) / m
    out = dict(estimate=n * math.log(sigma) + t, trace_res=t, sigma=sigma, c=c, gamma=gamma, xi=xi, d=d,
               taylor_terms=p_terms)
    if dg is not None:
        out["deg_g"] = dg
    return out


def logdet_hutchinson(A, lmin: float, lmax: float, degree: int, probes: int, seed: int,
                      kind: str = "rademacher", s_mode: str = "center", f32: bool = False, tol: float = 0.0) -> dict:
    """Eq. Léja8 over `probes` vectors of the G stream (the columns Algorithm 3 uses for G)."""
    if probes <= 0:
        raise ValueError("probes must be positive")
    G = _rng.probes(kind, seed, _rng.STREAM_G, A.n, probes)
    return hutchinson_logdet(A, lmin, lmax, degree, G, s_mode, f32, tol)


# ---------------------------------------------------------------------------------------------
# gradient of the frozen-basis estimator
# ---------------------------------------------------------------------------------------------

def _grad_values_uv(A, sigma: float, c: float, gamma: float, xi, d, V: np.ndarray, U: np.ndarray) -> np.ndarray:
    """d/d a_e of sum_j d_j <U, W_j> with W_0 = V, W_{j+1} = (B - xi_j I) W_j, U and V held fixed.

    Reverse recurrence: Lambda_m = d_m U, Lambda_j = d_j U + (B - xi_j I)^T Lambda_{j+1};
    dE/dB = sum_{j<m} Lambda_{j+1} W_j^T and dB/da_e = E_rc / (sigma gamma).
    """
    M = _scipy(A)
    MT = M.T.tocsr()
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    cols = np.asarray(A.colind, dtype=np.int64)
    m = len(d) - 1
    g = np.zeros(A.nnz)
    for col in range(V.shape[1]):
        Ws = [V[:, col].copy()]
        for j in range(m):
            w = Ws[-1]
            Ws.append(((M @ w) / sigma - c * w) / gamma - xi[j] * w)
        u = U[:, col]
        lam = d[m] * u
        for j in range(m - 1, -1, -1):
            g += lam[rows] * Ws[j][cols] / (sigma * gamma)
            lam = d[j] * u + (((MT @ lam) / sigma - c * lam) / gamma - xi[j] * lam)
    return g


def hutchpp_grad_values(A, lmin: float, lmax: float, degree: int, Q: np.ndarray, Gp: np.ndarray,
                        s_mode: str = "center") -> np.ndarray:
    """d E / d a_e for every stored entry e = (r, c) of A, where
    E(A) = n log sigma + sum_j d_j <U, W_j>,  U = [Q | Gp / k],  W_0 = [Q | Gp],
    W_{j+1} = (B - xi_j I) W_j,  B = (A / sigma - c I) / gamma,
    with Q, Gp, the bounds, sigma and d held fixed."""
    sigma = sigma_of(lmin)
    lt, ut = lmin / sigma, lmax / sigma
    xi, c, gamma, d, _ = newton_leja_setup(lt, ut, degree, s_mode)
    k = Gp.shape[1]
    V = np.concatenate([Q, Gp], axis=1)
    U = np.concatenate([Q, Gp / k], axis=1) if k > 0 else Q.copy()
    return _grad_values_uv(A, sigma, c, gamma, xi, d, V, U)


def hutchpp_qr_weights(A, lmin: float, lmax: float, degree: int, S: np.ndarray, G: np.ndarray,
                       s_mode: str = "center") -> dict:
    """The weights that carry the derivative of Algorithm 3's estimate through the sketch's QR.

    E = tr(F Pi) + (1/k) tr(F (I - Pi) G G^T (I - Pi)), Pi = Q Q^T the projector onto
    span(Y), Y = F S = Q R, F = p(A~). With the bounds, sigma and d fixed,
      dE = tr(dF [Pi + G' G'^T / k]) + tr(dPi Z),  Z = F - H (I - Pi) F - F (I - Pi) H,  H = G G^T / k,
      dPi = (I - Pi) dY Y^+ + (Y^+)^T dY^T (I - Pi),  Y^+ = R^-1 Q^T,  dY = dF S,
    so tr(dPi Z) = tr(Gamma^T dF S) with Gamma = 2 (I - Pi) Z Q R^-T, where
    Z Q = F Q - (1/k) G (G'^T F Q) - (1/k) (F G') (G^T Q).
    Returns Q, R, G', F Q, F G' and Gamma."""
    sigma = sigma_of(lmin)
    lt, ut = lmin / sigma, lmax / sigma
    xi, c, gamma, d, _ = newton_leja_setup(lt, ut, degree, s_mode)
    M = _scipy(A)
    k = G.shape[1]
    Y = leja_apply_columns(M, S, xi, d, c, gamma, sigma)
    Q, R = np.linalg.qr(Y, mode="reduced")
    Gp = G - Q @ (Q.T @ G)
    FQ = leja_apply_columns(M, Q, xi, d, c, gamma, sigma)
    FG = leja_apply_columns(M, Gp, xi, d, c, gamma, sigma)
    ZQ = FQ - G @ (Gp.T @ FQ) / k - FG @ (G.T @ Q) / k
    X = ZQ - Q @ (Q.T @ ZQ)
    Gamma = 2.0 * np.linalg.solve(R, X.T).T     # 2 X R^-T
    return dict(Q=Q, R=R, Gp=Gp, FQ=FQ, FG=FG, Gamma=Gamma, sigma=sigma, c=c, gamma=gamma, xi=xi, d=d)


def hutchpp_full_grad_values(A, lmin: float, lmax: float, degree: int, S: np.ndarray, G: np.ndarray,
                             s_mode: str = "center") -> np.ndarray:
    """d E / d a_e of Algorithm 3's estimate with Q = orth(p(A~) S) and G' = (I - QQ^T) G
    differentiated too (the bounds, sigma and d held fixed): the frozen-basis gradient plus the
    term sum_c Gamma_c^T (dF) S_c of hutchpp_qr_weights, by the same reverse recurrence with
    W_0 = S and U = Gamma."""
    w = hutchpp_qr_weights(A, lmin, lmax, degree, S, G, s_mode)
    g = hutchpp_grad_values(A, lmin, lmax, degree, w["Q"], w["Gp"], s_mode)
    return g + _grad_values_uv(A, w["sigma"], w["c"], w["gamma"], w["xi"], w["d"], S, w["Gamma"])


def frozen_estimate(A, values: np.ndarray, lmin: float, lmax: float, degree: int, Q: np.ndarray,
                    Gp: np.ndarray, s_mode: str = "center") -> float:
    """The frozen-basis estimator E evaluated with the stored values replaced by `values`."""
    sigma = sigma_of(lmin)
    lt, ut = lmin / sigma, lmax / sigma
    xi, c, gamma, d, _ = newton_leja_setup(lt, ut, degree, s_mode)
    M = sp.csr_matrix((np.asarray(values, dtype=np.float64), A.colind, A.rowptr), shape=(A.n, A.n))
    k = Gp.shape[1]
    FQ = leja_apply_columns(M, Q, xi, d, c, gamma, sigma)
    FG = leja_apply_columns(M, Gp, xi, d, c, gamma, sigma)
    return A.n * math.log(sigma) + float(np.sum(Q * FQ)) + float(np.sum(Gp * FG)) / k
