"""The log-determinant sweep along a pencil A(theta) = diag(D) + theta O (the theta grid of Section
5.3's GMRF maximum-likelihood experiment) on the GPU: every theta's estimate against the oracle on
the assembled matrix A(theta), and against ll_logdet_forward on the same matrix with the same
options (the sweep runs all thetas in one block pass pair, so only the rounding differs). Covers
the GMRF Q(theta) = I + theta Adj, a pencil with a varying diagonal D and a non-zero diagonal in O,
degrees that differ per theta (the block shrinks as thetas finish) in any input order, odd probe
widths (padded column groups), the plain Hutchinson estimator, one theta, a multi-tile size, and
the argument checks (needs a GB300 and the library)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from synth import CSR, gmrf_theta
from tests.gpu_util import TOL, lib, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


def _split_gmrf(N: int):
    """O = Adj (unit neighbour entries, stored zero diagonal) and D = 1 of Q(theta) = I + theta Adj."""
    A = gmrf_theta(N, 1.0)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    vals = np.where(np.asarray(A.colind) == rows, 0.0, 1.0)
    return CSR(A.n, A.rowptr, A.colind, vals), np.ones(A.n)


def _assemble(Om: CSR, D: np.ndarray, theta: float) -> CSR:
    """A(theta) = diag(D) + theta O on O's pattern (which stores every diagonal entry)."""
    rows = np.repeat(np.arange(Om.n), np.diff(Om.rowptr))
    vals = theta * np.asarray(Om.values, dtype=np.float64)
    diag = np.asarray(Om.colind) == rows
    assert np.array_equal(np.sort(rows[diag]), np.arange(Om.n))
    vals[diag] += D[rows[diag]]
    return CSR(Om.n, Om.rowptr, Om.colind, vals)


def _random_pencil(n: int, seed: int):
    """A symmetric O with a non-zero diagonal (a banded part and random far pairs, every diagonal
    entry stored) and D in [2, 3]: A(theta) is diagonally dominant for |theta| <= 0.25."""
    rng = np.random.default_rng(seed)
    ent = {}
    for i in range(n):
        ent[(i, i)] = rng.uniform(-0.5, 0.5)
        for off in (1, 3):
            if i + off < n:
                v = rng.uniform(-0.5, 0.5)
                ent[(i, i + off)] = v
                ent[(i + off, i)] = v
    for _ in range(n):
        i, j = rng.integers(0, n, 2)
        if i != j and (i, j) not in ent:
            v = rng.uniform(-0.5, 0.5)
            ent[(i, j)] = v
            ent[(j, i)] = v
    keys = sorted(ent)
    rows = np.array([k[0] for k in keys])
    cols = np.array([k[1] for k in keys], dtype=np.int32)
    vals = np.array([ent[k] for k in keys])
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    return CSR(n, rowptr, cols, vals), rng.uniform(2.0, 3.0, n)


def _run(L, h, Om, D, thetas, prec, probes, seed, degrees=None, est="hutchpp"):
    torch = need_gpu()
    dO = L.DeviceCSR.from_host(Om, "f32" if prec == "f32" else "f64")
    dD = torch.as_tensor(D, dtype=torch.float64).cuda()
    mats = [_assemble(Om, D, th) for th in thetas]
    bounds = [O.gershgorin(A) for A in mats]
    if degrees is None:
        degrees = [O.degree_from_bounds(lo, hi) for lo, hi in bounds]
    opts = L.options(degree=10, probes=probes, seed=seed, precision=prec, estimator=est)
    got = L.ll_logdet_sweep(h, dO, dD, thetas, bounds, opts, degrees=degrees)
    return got, mats, bounds, degrees, dO


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_gmrf_sweep_matches_oracle_and_forward(L, h, prec):
    """Q(theta) = I + theta Adj on a 48 x 48 grid, five thetas whose Gershgorin degrees run from 20
    to 48, given out of degree order."""
    Om, D = _split_gmrf(48)
    thetas = [-0.22, -0.24, -0.20, 0.15, -0.23]
    got, mats, bounds, degrees, _ = _run(L, h, Om, D, thetas, prec, 30, 4)
    assert len(set(degrees)) >= 4
    for g, th in enumerate(thetas):
        A = mats[g]
        lo, hi = bounds[g]
        want = O.logdet_leja(A, lo, hi, degrees[g], 30, 4, f32=(prec == "f32"))["estimate"]
        assert abs(got[g] - want) <= TOL[prec] * abs(want), (th, got[g], want)
        dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
        one = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=degrees[g], probes=30, seed=4, precision=prec))
        assert abs(got[g] - one) <= (1e-12 if prec != "f32" else TOL["f32"]) * abs(one), (th, got[g], one)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_pencil_with_varying_diagonal(L, h, prec):
    """D varies per row and O has diagonal entries: the row shift s2 D_r + beta and the scaled row
    sums are both exercised (the GMRF's D = 1 would not tell rows apart). k = 11 (odd: padded
    column groups), and an explicit degree list."""
    Om, D = _random_pencil(3001, seed=5)
    thetas = [0.25, -0.1, 0.05]
    degrees = [14, 31, 9]
    got, mats, bounds, degrees, _ = _run(L, h, Om, D, thetas, prec, 33, 2, degrees=degrees)
    for g in range(len(thetas)):
        lo, hi = bounds[g]
        want = O.logdet_leja(mats[g], lo, hi, degrees[g], 33, 2, f32=(prec == "f32"))["estimate"]
        assert abs(got[g] - want) <= TOL[prec] * abs(want), (thetas[g], got[g], want)


def test_sweep_hutchinson_and_single_theta(L, h):
    Om, D = _split_gmrf(40)
    thetas = [-0.21, 0.1]
    got, mats, bounds, degrees, _ = _run(L, h, Om, D, thetas, "df64", 16, 9, est="hutchinson")
    for g in range(2):
        lo, hi = bounds[g]
        want = O.logdet_hutchinson(mats[g], lo, hi, degrees[g], 16, 9)["estimate"]
        assert abs(got[g] - want) <= TOL["df64"] * abs(want)
    one, mats, bounds, degrees, _ = _run(L, h, Om, D, [-0.2], "df64", 24, 3)
    lo, hi = bounds[0]
    want = O.logdet_leja(mats[0], lo, hi, degrees[0], 24, 3)["estimate"]
    assert abs(one[0] - want) <= TOL["df64"] * abs(want)


@pytest.mark.parametrize("prec", ["df64", "f32"])
def test_gmrf_sweep_multi_tile(L, h, prec):
    """A 330 x 330 grid (108,900 rows: many tiles per CTA), five thetas, against the forward."""
    Om, D = _split_gmrf(330)
    thetas = [-0.24, -0.23, -0.22, -0.21, -0.20]
    got, mats, bounds, degrees, _ = _run(L, h, Om, D, thetas, prec, 30, 0)
    info = h.info()
    assert info["kernel_pass2"] == L.LL_KERNEL_TMA and info["deg_max_pass2"] == max(degrees)
    for g in range(len(thetas)):
        lo, hi = bounds[g]
        dA = L.DeviceCSR.from_host(mats[g], "f32" if prec == "f32" else "f64")
        one = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=degrees[g], probes=30, seed=0, precision=prec))
        assert abs(got[g] - one) <= (1e-12 if prec != "f32" else TOL["f32"]) * abs(one), (thetas[g], got[g], one)


def test_sweep_many_thetas(L, h):
    """Twelve thetas of 20 columns (240 trace columns, few rows per tile), against the forward."""
    Om, D = _split_gmrf(60)
    thetas = [-0.23 + 0.04 * k for k in range(12)]   # (no theta = 0: A = I has lmin = lmax)
    got, mats, bounds, degrees, _ = _run(L, h, Om, D, thetas, "df64", 30, 1)
    for g in (0, 5, 11):
        lo, hi = bounds[g]
        dA = L.DeviceCSR.from_host(mats[g])
        one = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=degrees[g], probes=30, seed=1))
        assert abs(got[g] - one) <= 1e-12 * abs(one), (thetas[g], got[g], one)


def test_sweep_argument_checks(L, h):
    torch = need_gpu()
    Om, D = _split_gmrf(20)
    dO = L.DeviceCSR.from_host(Om)
    dD = torch.ones(Om.n, dtype=torch.float64, device="cuda")
    b = [(0.2, 1.8)]
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_sweep(h, dO, dD, [-0.2], b, L.options(degree=10, probes=30, tol=1e-6))
    assert ei.value.name == "LL_ERR_UNSUPPORTED"
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_sweep(h, dO, dD, [-0.2], b, L.options(degree=10, probes=30, keep_for_backward=True))
    assert ei.value.name == "LL_ERR_UNSUPPORTED"
    # 52 thetas of 20 columns: more than 1024 trace columns
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_sweep(h, dO, dD, [-0.2] * 52, b * 52, L.options(degree=10, probes=30))
    assert ei.value.name == "LL_ERR_UNSUPPORTED"
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_sweep(h, dO, dD, [-0.2], [(0.0, 1.8)], L.options(degree=10, probes=30))
    assert ei.value.name == "LL_ERR_BAD_BOUNDS"
    with pytest.raises(ValueError):
        L.ll_logdet_sweep(h, dO, dD[:-1].contiguous(), [-0.2], b, L.options(degree=10, probes=30))
