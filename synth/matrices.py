"""Seeded sparse SPD test matrices in CSR form (int32 row pointers and column indices, float64
values, column indices ascending within each row).

The families are the synthetic GMRF precision matrices used as workloads for the Léja-point
log-determinant estimator (arXiv 2603.02207, Section 5): shifted Dirichlet Laplacians on 2-D and
3-D grids, a Matérn-type operator tau*(kappa^2 I + L)^2, batches of shifted 2-D Laplacians with
random sizes and shifts, the Laplacian of a random power-law graph, and the paper's own
pentadiagonal family (Section 5.1). Nothing here depends on the estimator.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class CSR:
    """A square sparse matrix in CSR layout.

    rowptr: int32[n+1], colind: int32[nnz] (ascending within a row), values: float64[nnz].
    """

    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    values: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.values, self.colind, self.rowptr), shape=(self.n, self.n))

    @staticmethod
    def from_scipy(m) -> "CSR":
        m = sp.csr_matrix(m)
        m.sum_duplicates()
        m.sort_indices()
        n = m.shape[0]
        if m.nnz >= 2**31 or n >= 2**31:
            raise ValueError("matrix too large for int32 CSR indices")
        return CSR(n=n,
                   rowptr=np.ascontiguousarray(m.indptr, dtype=np.int32),
                   colind=np.ascontiguousarray(m.indices, dtype=np.int32),
                   values=np.ascontiguousarray(m.data, dtype=np.float64))


def _path_laplacian(N: int) -> sp.csr_matrix:
    """1-D Dirichlet Laplacian tridiag(-1, 2, -1) of order N."""
    e = np.ones(N)
    return sp.diags([-e[:-1], 2.0 * e, -e[:-1]], [-1, 0, 1], format="csr")


def laplacian_2d(N: int, shift: float = 0.0) -> CSR:
    """5-point Dirichlet Laplacian on an N x N grid (lexicographic order) plus shift*I.

    Diagonal 4 + shift, -1 for each existing grid neighbour; n = N^2, nnz = 5N^2 - 4N.
    Eigenvalues 4 sin^2(i pi / (2(N+1))) + 4 sin^2(j pi / (2(N+1))) + shift.
    """
    I = sp.identity(N, format="csr")
    T = _path_laplacian(N)
    L = sp.kron(I, T, format="csr") + sp.kron(T, I, format="csr")
    return CSR.from_scipy(L + shift * sp.identity(N * N, format="csr"))


def laplacian_3d(N: int, shift: float = 0.0) -> CSR:
    """7-point Dirichlet Laplacian on an N^3 grid plus shift*I; nnz = 7N^3 - 6N^2."""
    I = sp.identity(N, format="csr")
    T = _path_laplacian(N)
    II = sp.kron(I, I, format="csr")
    L = (sp.kron(II, T, format="csr") + sp.kron(sp.kron(I, T, format="csr"), I, format="csr")
         + sp.kron(T, II, format="csr"))
    return CSR.from_scipy(L + shift * sp.identity(N ** 3, format="csr"))


def _matern_K(N: int, kappa: float) -> sp.csr_matrix:
    I = sp.identity(N, format="csr")
    T = _path_laplacian(N)
    L = sp.kron(I, T, format="csr") + sp.kron(T, I, format="csr")
    return (L + (kappa * kappa) * sp.identity(N * N, format="csr")).tocsr()


def matern_2d(N: int, kappa: float, tau: float) -> CSR:
    """Matérn-type GMRF precision tau * (kappa^2 I + L_2D)^2 on an N x N grid (13-point stencil).

    Formed as the exact sparse product K @ K with K = kappa^2 I + L_2D, so that its eigenvalues
    are tau * (kappa^2 + mu_ij)^2 with mu_ij the 2-D Laplacian eigenvalues.
    """
    K = _matern_K(N, kappa)
    return CSR.from_scipy(tau * (K @ K))


def matern_2d_derivatives(N: int, kappa: float, tau: float) -> tuple[np.ndarray, np.ndarray]:
    """Entrywise derivatives of matern_2d(N, kappa, tau) values with respect to (kappa, tau),
    aligned with its CSR pattern: dQ/dkappa = 4 kappa tau (kappa^2 I + L), dQ/dtau = K^2."""
    K = _matern_K(N, kappa)
    Q = CSR.from_scipy(tau * (K @ K))
    K2 = CSR.from_scipy(K @ K)
    assert np.array_equal(K2.colind, Q.colind) and np.array_equal(K2.rowptr, Q.rowptr)
    dK = (4.0 * kappa * tau) * K
    dK = sp.csr_matrix(dK)
    dk_vals = np.zeros(Q.nnz)
    # scatter the 5-point values of 4 kappa tau K into the 13-point pattern
    Qs = Q.to_scipy()
    dKc = dK.tocoo()
    lookup = sp.csr_matrix((np.arange(1, Q.nnz + 1, dtype=np.float64), Q.colind, Q.rowptr), shape=Qs.shape)
    pos = np.asarray(lookup[dKc.row, dKc.col]).ravel().astype(np.int64) - 1
    assert (pos >= 0).all()
    dk_vals[pos] = dKc.data
    return dk_vals, K2.values.copy()


def gmrf_batch_params(count: int = 64, seed: int = 2, side_lo: int = 64, side_hi: int = 512,
                      tau_lo: float = 0.01, tau_hi: float = 1.0) -> list[tuple[int, float]]:
    """(side, tau) for a batch of shifted 2-D Laplacians L_2D + tau I.

    Draw 2i gives side_i = round(exp(U[ln side_lo, ln side_hi])), draw 2i+1 gives
    tau_i = U[tau_lo, tau_hi]; both from numpy's PCG64 stream with the given seed.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        u = rng.random()
        side = int(round(math.exp(math.log(side_lo) + u * (math.log(side_hi) - math.log(side_lo)))))
        t = rng.random()
        tau = tau_lo + t * (tau_hi - tau_lo)
        out.append((side, tau))
    return out


def powerlaw_laplacian(n: int, mean_degree: float = 16.0, beta: float = 2.3, seed: int = 3,
                       shift: float = 1e-2, w_lo: float = 0.5, w_hi: float = 1.5, device=None) -> CSR:
    """Weighted Laplacian (D - W) + shift*I of a Chung-Lu random graph with power-law degrees.

    Expected degrees w_i proportional to (i+1)^(-1/(beta-1)), rescaled to the requested mean and
    capped at sqrt(sum w). mean_degree*n/2 endpoint pairs are drawn with probability
    proportional to w (inverse CDF of uniform draws); self-loops are dropped, repeated pairs are
    merged into one edge, each edge gets a weight U[w_lo, w_hi], and vertices are relabelled by a
    random permutation. Degrees are summed per vertex in edge order (bincount), and the CSR lists
    each row's entries by ascending column.

    device: None runs everything in NumPy; a torch device (e.g. "cuda") runs the inverse-CDF
    search, the duplicate merge and the CSR sort there. The random draws come from the same NumPy
    generator and the degree sums are taken on the host in the same order, so both give the same
    CSR bit for bit; the device path only makes the n = 2^22 instance quick to build.
    """
    rng = np.random.default_rng(seed)
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (beta - 1.0))
    w *= mean_degree * n / w.sum()
    w = np.minimum(w, math.sqrt(w.sum()))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    n_pairs = int(round(mean_degree * n / 2))
    r1 = rng.random(n_pairs)
    r2 = rng.random(n_pairs)
    if device is None:
        u = np.searchsorted(cdf, r1, side="right")
        v = np.searchsorted(cdf, r2, side="right")
        np.minimum(u, n - 1, out=u)
        np.minimum(v, n - 1, out=v)
        keep = u != v
        u, v = u[keep], v[keep]
        lo = np.minimum(u, v).astype(np.int64)
        hi = np.maximum(u, v).astype(np.int64)
        key = np.unique(lo * n + hi)
    else:
        import torch
        tc = torch.from_numpy(cdf).to(device)
        u = torch.searchsorted(tc, torch.from_numpy(r1).to(device), right=True).clamp_(max=n - 1)
        v = torch.searchsorted(tc, torch.from_numpy(r2).to(device), right=True).clamp_(max=n - 1)
        keep = u != v
        u, v = u[keep], v[keep]
        tkey = torch.unique(torch.minimum(u, v) * n + torch.maximum(u, v), sorted=True)
        key = tkey.cpu().numpy()
        del u, v, keep, tc
    lo, hi = key // n, key % n
    wt = w_lo + (w_hi - w_lo) * rng.random(key.shape[0])
    perm = rng.permutation(n)
    lo, hi = perm[lo], perm[hi]
    deg = np.bincount(lo, weights=wt, minlength=n) + np.bincount(hi, weights=wt, minlength=n)
    diag = np.arange(n, dtype=np.int64)
    rows = np.concatenate([lo, hi, diag])
    cols = np.concatenate([hi, lo, diag])
    vals = np.concatenate([-wt, -wt, deg + shift])
    if device is None:
        order = np.argsort(rows * n + cols, kind="stable")
        rows, cols, vals = rows[order], cols[order], vals[order]
    else:
        import torch
        tr = torch.from_numpy(rows).to(device)
        tcl = torch.from_numpy(cols).to(device)
        order = torch.argsort(tr * n + tcl)
        rows = tr[order].cpu().numpy()
        cols = tcl[order].cpu().numpy()
        vals = torch.from_numpy(vals).to(device)[order].cpu().numpy()
        del tr, tcl, order
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return CSR(n=n, rowptr=rowptr.astype(np.int32), colind=cols.astype(np.int32), values=vals)


def pentadiagonal(n: int, seed: int = 0) -> CSR:
    """The paper's synthetic pentadiagonal SPD family (Section 5.1): the five diagonals at
    offsets 0, +1, +2, -1, -2 are U[0,1] samples, then Q <- Q + Q^T + n I."""
    rng = np.random.default_rng(seed)
    diags = [rng.random(n), rng.random(n - 1), rng.random(n - 2), rng.random(n - 1), rng.random(n - 2)]
    Q = sp.diags(diags, [0, 1, 2, -1, -2], format="csr")
    Q = Q + Q.T + n * sp.identity(n, format="csr")
    return CSR.from_scipy(Q)


def gmrf_theta(N: int, theta: float) -> CSR:
    """Precision matrix Q(theta) = I + theta * Adj of the 4-neighbour GMRF on an N x N grid
    (lexicographic order; Adj the grid graph's adjacency: 1 for each existing neighbour), the
    model of the paper's maximum-likelihood experiment (Section 5.3, "partial correlation"
    theta). Eigenvalues 1 + theta (a_i + a_j), a_i = 2 cos(i pi / (N + 1)); SPD for |theta| < 1/4.
    Built directly in CSR (no sparse products), so N = 5000 (n = 2.5e7) takes seconds."""
    n = N * N
    j = np.tile(np.arange(N, dtype=np.int32), N)
    r = np.arange(n, dtype=np.int32)
    offs = np.array([-N, -1, 0, 1, N], dtype=np.int32)   # ascending column order within a row
    valid = np.empty((n, 5), dtype=bool)
    valid[:, 0] = r >= N
    valid[:, 1] = j > 0
    valid[:, 2] = True
    valid[:, 3] = j < N - 1
    valid[:, 4] = r < n - N
    cols = r[:, None] + offs[None, :]
    colind = cols[valid]
    vals = np.where(offs == 0, 1.0, theta)
    values = np.broadcast_to(vals, (n, 5))[valid]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(valid.sum(axis=1), out=rowptr[1:])
    return CSR(n=n, rowptr=rowptr.astype(np.int32), colind=np.ascontiguousarray(colind, dtype=np.int32),
               values=np.ascontiguousarray(values, dtype=np.float64))


def diagonal(d: np.ndarray) -> CSR:
    """Diagonal matrix diag(d)."""
    d = np.asarray(d, dtype=np.float64)
    n = d.shape[0]
    return CSR(n=n, rowptr=np.arange(n + 1, dtype=np.int32), colind=np.arange(n, dtype=np.int32), values=d.copy())


def random_spd(n: int, nnz_per_row: int = 6, seed: int = 0, shift: float = 0.5,
               empty_rows: int = 0, dense_row: bool = False) -> CSR:
    """Random sparse symmetric, strictly diagonally dominant matrix (hence SPD).

    Off-diagonal entries are U[-1, 1]; the diagonal is the row's absolute off-diagonal sum plus
    shift*(1 + U[0,1]). `empty_rows` rows (and columns) carry only their diagonal entry;
    `dense_row` couples row 0 to every other row.
    """
    rng = np.random.default_rng(seed)
    m = max(0, n * nnz_per_row // 2)
    r = rng.integers(0, n, m)
    c = rng.integers(0, n, m)
    v = rng.uniform(-1.0, 1.0, m)
    if dense_row and n > 1:
        r = np.concatenate([r, np.zeros(n - 1, dtype=r.dtype)])
        c = np.concatenate([c, np.arange(1, n, dtype=c.dtype)])
        v = np.concatenate([v, rng.uniform(-1.0, 1.0, n - 1) * 0.1])
    keep = r != c
    if empty_rows > 0:
        iso = rng.choice(n, size=min(empty_rows, n), replace=False)
        mask = np.ones(n, dtype=bool)
        mask[iso] = False
        keep &= mask[r] & mask[c]
    r, c, v = r[keep], c[keep], v[keep]
    W = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    W = W + W.T
    rowsum = np.asarray(abs(W).sum(axis=1)).ravel()
    diag = rowsum + shift * (1.0 + rng.random(n))
    return CSR.from_scipy(W + sp.diags(diag, 0, format="csr"))


def csr_from_dense(M: np.ndarray) -> CSR:
    return CSR.from_scipy(sp.csr_matrix(np.asarray(M, dtype=np.float64)))
