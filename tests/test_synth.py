"""Seeded input generators (CPU): the power-law generator's NumPy and torch back ends agree bit
for bit, and its output is a valid Laplacian-plus-shift CSR."""
from __future__ import annotations

import numpy as np
import pytest

from synth import powerlaw_laplacian


def test_powerlaw_backends_agree_bitwise():
    torch = pytest.importorskip("torch")
    a = powerlaw_laplacian(1 << 12, seed=3)
    b = powerlaw_laplacian(1 << 12, seed=3, device=torch.device("cpu"))
    assert np.array_equal(a.rowptr, b.rowptr)
    assert np.array_equal(a.colind, b.colind)
    assert np.array_equal(a.values, b.values)


def test_powerlaw_is_a_shifted_laplacian():
    A = powerlaw_laplacian(1 << 13, seed=5, shift=1e-2)
    S = A.to_scipy()
    assert (abs(S - S.T)).max() == 0.0
    rows = np.asarray(S.sum(axis=1)).ravel()
    assert np.allclose(rows, 1e-2, atol=1e-9)
    d = S.diagonal()
    off = S - __import__("scipy.sparse", fromlist=["diags"]).diags(d)
    assert off.max() <= 0.0
    assert np.all(np.diff(A.rowptr) >= 1)
    for r in range(0, A.n, 997):
        c = A.colind[A.rowptr[r]:A.rowptr[r + 1]]
        assert np.all(np.diff(c) > 0)
    # mean stored entries per row about mean degree + 1 (duplicates merged)
    assert 12.0 < A.nnz / A.n < 17.5


def test_pentadiagonal_family():
    """Section 5.1's synthetic matrices: symmetric, entries within two of the diagonal, diagonal
    dominant with the n I shift, seeded."""
    from synth import pentadiagonal
    A = pentadiagonal(500, seed=4)
    M = A.to_scipy()
    assert (abs(M - M.T)).max() == 0.0
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    assert np.abs(A.colind - rows).max() == 2
    assert A.nnz == 5 * A.n - 6
    d = M.diagonal()
    off = np.asarray(abs(M).sum(axis=1)).ravel() - d
    assert np.all(d - off > 0) and d.min() >= A.n
    B = pentadiagonal(500, seed=4)
    assert np.array_equal(A.values, B.values) and not np.array_equal(A.values, pentadiagonal(500, seed=5).values)


def test_gmrf_theta_matches_kronecker_form():
    """The direct CSR construction equals I + theta (Adj_path (x) I + I (x) Adj_path)."""
    import scipy.sparse as sp
    from synth import gmrf_theta
    for N, theta in ((1, -0.22), (2, 0.1), (9, -0.22), (16, 0.24)):
        A = gmrf_theta(N, theta)
        e = np.ones(N)
        P = sp.diags([e[:-1], e[:-1]], [-1, 1], shape=(N, N), format="csr")
        I = sp.identity(N, format="csr")
        ref = (sp.identity(N * N) + theta * (sp.kron(P, I) + sp.kron(I, P))).tocsr()
        ref.eliminate_zeros()
        ref.sort_indices()
        assert np.array_equal(A.rowptr, ref.indptr) and np.array_equal(A.colind, ref.indices)
        assert np.array_equal(A.values, ref.data)
        assert A.rowptr.dtype == np.int32 and A.colind.dtype == np.int32
