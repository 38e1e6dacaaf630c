"""The degree-ordered forward (ll_options.reorder): the passes run on P A P^T with the rows ordered
by entry count and the probe rows keeping their original rows' values, so the estimate equals the
unpermuted one up to the order of its sums. Checked against the unpermuted forward and the oracle
on power-law graph Laplacians, with Hutch++ and Hutchinson, in every precision; the automatic
choice (power-law graph: on; stencil: off; with keep_for_backward: off); the structure cache
(a structure rewritten in place under the same pointers is reordered afresh); graph replay
(needs a GB300 and the library)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from synth import CSR, laplacian_3d, powerlaw_laplacian
from tests.gpu_util import TOL, lib, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


def _bounds(A):
    lo, hi = O.gershgorin(A)
    return 0.01, hi


def _relabel(A: CSR, seed: int) -> CSR:
    """P A P^T for a random permutation: the same n and nnz, another structure."""
    rng = np.random.default_rng(seed)
    n = A.n
    p = rng.permutation(n)                      # new label of old row i
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    nr, nc = p[rows], p[np.asarray(A.colind)]
    order = np.lexsort((nc, nr))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rowptr, nr + 1, 1)
    return CSR(n, np.cumsum(rowptr).astype(np.int32), nc[order].astype(np.int32), np.asarray(A.values)[order])


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("est", ["hutchpp", "hutchinson"])
def test_degree_order_matches_the_matrix_order_and_the_oracle(L, prec, est):
    A = powerlaw_laplacian(1 << 13, seed=5)
    lo, hi = _bounds(A)
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    h = L.Handle()
    got = {}
    for r in ("none", "degree"):
        got[r] = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=30, probes=30, seed=2, precision=prec,
                                                              estimator=est, reorder=r))
        assert h.info()["reordered"] == (r == "degree")
    # each row's arithmetic is the same in either order (its entries keep their order); only the
    # sums across rows (traces, Grams) are reordered
    tol_same = 1e-12 if prec != "f32" else 1e-9
    assert abs(got["degree"] - got["none"]) <= tol_same * abs(got["none"])
    f = O.logdet_leja if est == "hutchpp" else O.logdet_hutchinson
    want = f(A, lo, hi, 30, 30, 2, f32=(prec == "f32"))["estimate"]
    assert abs(got["degree"] - want) <= TOL[prec] * abs(want)


def test_automatic_order_choice(L):
    h = L.Handle()
    P = powerlaw_laplacian(1 << 14, seed=7)
    dP = L.DeviceCSR.from_host(P)
    lo, hi = _bounds(P)
    e_auto = L.ll_logdet_forward(h, dP, lo, hi, L.options(degree=20, probes=30, seed=1))
    assert h.info()["reordered"] == 1
    e_none = L.ll_logdet_forward(h, dP, lo, hi, L.options(degree=20, probes=30, seed=1, reorder="none"))
    assert abs(e_auto - e_none) <= 1e-12 * abs(e_none)
    # kept for a backward: the matrix's order
    L.ll_logdet_forward(h, dP, lo, hi, L.options(degree=20, probes=30, seed=1, keep_for_backward=True))
    assert h.info()["reordered"] == 0
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_forward(h, dP, lo, hi, L.options(degree=20, probes=30, seed=1, keep_for_backward=True,
                                                     reorder="degree"))
    assert ei.value.name == "LL_ERR_UNSUPPORTED"
    # a stencil: the matrix's order
    S = laplacian_3d(24, 0.05)
    L.ll_logdet_forward(h, L.DeviceCSR.from_host(S), 0.05, 12.05, L.options(degree=10, probes=30))
    assert h.info()["reordered"] == 0


def test_structure_rewritten_in_place_is_reordered_afresh(L):
    """Same device pointers, another structure of the same size: the checksum tells it from the
    cached one, and the estimate equals a fresh handle's on the new structure."""
    torch = need_gpu()
    A = powerlaw_laplacian(1 << 13, seed=11)
    B = _relabel(A, seed=3)
    lo, hi = _bounds(A)
    dA = L.DeviceCSR.from_host(A)
    h = L.Handle()
    # (fixed kernels: the autotuners time candidates and may choose differently per handle)
    o = L.options(degree=25, probes=30, seed=4, reorder="degree", step_kernel="tma", qr_gram="dfloat")
    ea = L.ll_logdet_forward(h, dA, lo, hi, o)
    dA.rowptr.copy_(torch.as_tensor(np.asarray(B.rowptr, dtype=np.int32)))
    dA.colind.copy_(torch.as_tensor(np.asarray(B.colind, dtype=np.int32)))
    dA.values.copy_(torch.as_tensor(np.asarray(B.values)))
    eb = L.ll_logdet_forward(h, dA, lo, hi, o)
    fresh = L.ll_logdet_forward(L.Handle(), L.DeviceCSR.from_host(B), lo, hi, o)
    assert eb == fresh
    # each against the oracle on its own structure (B's probes follow B's rows)
    for est, M in ((ea, A), (eb, B)):
        want = O.logdet_leja(M, lo, hi, 25, 30, 4)["estimate"]
        assert abs(est - want) <= TOL["df64"] * abs(want)


def test_degree_order_graph_replay_and_values_in_place(L):
    torch = need_gpu()
    A = powerlaw_laplacian(1 << 13, seed=13)
    lo, hi = _bounds(A)
    dA = L.DeviceCSR.from_host(A)
    h = L.Handle()
    o = L.options(degree=20, probes=30, seed=6, reorder="degree", use_graph=True)
    e1 = L.ll_logdet_forward(h, dA, lo, hi, o)
    e2 = L.ll_logdet_forward(h, dA, lo, hi, o)   # replay
    assert e1 == e2
    # new values under the same structure: gathered afresh through the cached order
    dA.values.mul_(2.0)
    e3 = L.ll_logdet_forward(h, dA, 2 * lo, 2 * hi, o)
    ref = L.ll_logdet_forward(h, dA, 2 * lo, 2 * hi, L.options(degree=20, probes=30, seed=6, reorder="none"))
    assert abs(e3 - ref) <= 1e-12 * abs(ref)
    assert abs(e3 - (e1 + A.n * np.log(2.0))) <= 1e-9 * abs(e3)
