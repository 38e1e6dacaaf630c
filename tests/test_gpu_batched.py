"""Batched persistent launch (many GMRFs of uneven size) against single-matrix estimates and the
oracle (needs a GB300)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from synth import gmrf_batch_params, laplacian_2d, random_spd
from tests.gpu_util import TOL, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


def _batch(scale=8, count=9, seed=2):
    params = gmrf_batch_params(count=count, seed=seed, side_lo=64 // scale, side_hi=512 // scale)
    mats = [laplacian_2d(side, tau) for side, tau in params]
    bounds = [(tau, 8.0 + tau) for _, tau in params]
    return mats, bounds


@pytest.mark.parametrize("prec", ["df64", "f32", "f64"])
def test_batched_matches_oracle(L, h, prec):
    mats, bounds = _batch()
    dm = [L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64") for A in mats]
    opts = L.options(probes=30, seed=5, precision=prec)
    got = L.ll_logdet_batched(h, dm, bounds, opts)
    for i, (A, (lo, hi)) in enumerate(zip(mats, bounds)):
        sigma = O.sigma_of(lo)
        m = O.degree_from_bounds(lo / sigma, hi / sigma)
        want = O.logdet_leja(A, lo, hi, m, 30, 5 + i)["estimate"]
        assert abs(got[i] - want) / abs(want) < TOL[prec], (i, got[i], want)


def test_batched_matches_single_matrix_calls(L, h):
    mats, bounds = _batch(scale=4, count=12, seed=7)
    dm = [L.DeviceCSR.from_host(A) for A in mats]
    degrees = [10 + 7 * i for i in range(len(mats))]
    got = L.ll_logdet_batched(h, dm, bounds, L.options(probes=24, seed=1, precision="df64"), degrees=degrees)
    for i, A in enumerate(dm):
        single = L.ll_logdet_forward(h, A, *bounds[i], L.options(degree=degrees[i], probes=24, seed=1 + i, precision="df64"))
        assert got[i] == pytest.approx(single, rel=1e-12)


def test_batched_irregular_matrices(L, h):
    mats = [random_spd(n, seed=n, empty_rows=2, dense_row=(n % 2 == 0)) for n in (300, 517, 1000, 77)]
    bounds = []
    for A in mats:
        lo, hi = O.gershgorin(A)
        bounds.append((max(lo, 0.05), hi))
    dm = [L.DeviceCSR.from_host(A) for A in mats]
    got = L.ll_logdet_batched(h, dm, bounds, L.options(probes=15, seed=3, precision="df64"), degrees=[20, 25, 30, 35])
    for i, A in enumerate(mats):
        want = O.logdet_leja(A, *bounds[i], [20, 25, 30, 35][i], 15, 3 + i)["estimate"]
        assert abs(got[i] - want) / abs(want) < 1e-10


def test_batched_wait_timeout_is_reported(L, h):
    """A zero spin budget makes every dependency wait that is not already satisfied give up at
    once: the call reports LL_ERR_TIMEOUT, nothing hangs, and the handle keeps working."""
    mats, bounds = _batch(scale=2, count=6, seed=3)
    dm = [L.DeviceCSR.from_host(A) for A in mats]
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_batched(h, dm, bounds, L.options(probes=30, seed=1, timeout_cycles=1))
    assert ei.value.name == "LL_ERR_TIMEOUT"
    est = L.ll_logdet_batched(h, dm[:2], bounds[:2], L.options(probes=30, seed=1))
    assert np.all(np.isfinite(est))


def test_batched_graph_replay(L, h):
    """An identical batched call replays the captured device work: same estimates as the eager
    call and as a handle without graphs; changed bounds capture anew."""
    mats, bounds = _batch()
    dm = [L.DeviceCSR.from_host(A) for A in mats]
    opts = L.options(probes=9, seed=6)
    e1 = L.ll_logdet_batched(h, dm, bounds, opts)
    l1 = h.info()["kernel_launches"]
    e2 = L.ll_logdet_batched(h, dm, bounds, opts)
    i2 = h.info()
    assert np.array_equal(e1, e2)
    assert i2["kernel_launches"] == l1 and i2["ms_pass2"] > 0
    # a second handle tunes the launch shape on its own: the tiles (and so the order of the trace
    # sums) may differ, the estimates only to rounding
    h2 = L.Handle()
    e3 = L.ll_logdet_batched(h2, dm, bounds, L.options(probes=9, seed=6, use_graph=False))
    np.testing.assert_allclose(e1, e3, rtol=1e-12)
    b2 = [(lo, hi * 1.5) for lo, hi in bounds]
    e4 = L.ll_logdet_batched(h, dm, b2, opts)
    e5 = L.ll_logdet_batched(h2, dm, b2, L.options(probes=9, seed=6, use_graph=False))
    np.testing.assert_allclose(e4, e5, rtol=1e-12)
    assert not np.array_equal(e4, e1)


@pytest.mark.parametrize("prec", ["df64", "f32", "f64"])
def test_batched_tma_matches_register_kernel(L, prec):
    """The TMA-fed persistent passes and the register-gather persistent passes run the same per-row
    arithmetic: estimates agree to the rounding of the trace sums (tiles differ in size, so the
    per-tile partials are summed in a different order). Many small matrices of uneven degree keep
    several matrices and steps in flight in every CTA."""
    params = gmrf_batch_params(count=24, seed=11, side_lo=12, side_hi=96)
    mats = [laplacian_2d(side, tau) for side, tau in params]
    bounds = [(tau, 8.0 + tau) for _, tau in params]
    dm = [L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64") for A in mats]
    res = {}
    for kernel in ("gather", "tma"):
        h = L.Handle()
        est = L.ll_logdet_batched(h, dm, bounds, L.options(probes=30, seed=4, precision=prec, step_kernel=kernel))
        res[kernel] = (est, h.info())
    assert res["gather"][1]["kernel_pass1"] == L.LL_KERNEL_GATHER
    assert res["tma"][1]["kernel_pass1"] == L.LL_KERNEL_TMA and res["tma"][1]["kernel_pass2"] == L.LL_KERNEL_TMA
    np.testing.assert_allclose(res["tma"][0], res["gather"][0], rtol=1e-12 if prec != "f32" else 1e-9)
    # auto runs the shape its autotuner picked (either kernel): the same estimates to rounding
    h = L.Handle()
    est = L.ll_logdet_batched(h, dm, bounds, L.options(probes=30, seed=4, precision=prec))
    assert h.info()["batch_tuned"] == 1
    np.testing.assert_allclose(est, res["tma"][0], rtol=1e-12 if prec != "f32" else 1e-9)
    for i in (0, 7, 23):
        A, (lo, hi) = mats[i], bounds[i]
        sigma = O.sigma_of(lo)
        m = O.degree_from_bounds(lo / sigma, hi / sigma)
        want = O.logdet_leja(A, lo, hi, m, 30, 4 + i, f32=(prec == "f32"))["estimate"]
        assert abs(res["tma"][0][i] - want) / abs(want) < TOL[prec], (i, res["tma"][0][i], want)


def test_batched_tma_stall_timeout_is_reported(L):
    """The stall hook leaves the first tile of one CTA incomplete (16 expected bytes no copy
    delivers): its consumers give up, the other CTAs stop at their next dependency on it, every
    CTA drains its copies and returns, the call reports LL_ERR_TIMEOUT and the handle stays usable."""
    mats, bounds = _batch(scale=4, count=5, seed=9)
    dm = [L.DeviceCSR.from_host(A) for A in mats]
    h = L.Handle()
    h.debug_inject("stall")
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_batched(h, dm, bounds, L.options(probes=30, seed=1, timeout_cycles=1_000_000, use_graph=False,
                                                     step_kernel="tma"))
    assert ei.value.name == "LL_ERR_TIMEOUT"
    h.debug_inject("none")
    a = L.ll_logdet_batched(h, dm, bounds, L.options(probes=30, seed=1, step_kernel="tma"))
    b = L.ll_logdet_batched(L.Handle(), dm, bounds, L.options(probes=30, seed=1, step_kernel="gather"))
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_batched_autotuner_choice_is_cached_and_reported(L):
    """LL_KERNEL_AUTO: the first call for a batch shape times the TMA passes with 512, 384 and 256
    consumer threads and the register kernel, and keeps the fastest shape of each pass; a second
    call of the same shape runs it directly (no tuning launches) with the same estimates. An
    explicit kernel is not tuned."""
    mats, bounds = _batch(scale=4, count=10, seed=12)
    dm = [L.DeviceCSR.from_host(A) for A in mats]
    h = L.Handle()
    opts = L.options(probes=30, seed=2, use_graph=False)
    e1 = L.ll_logdet_batched(h, dm, bounds, opts)
    i1 = h.info()
    assert i1["batch_tuned"] == 1
    assert i1["threads_pass1"] > 0 and i1["threads_pass2"] > 0
    if i1["kernel_pass1"] == L.LL_KERNEL_TMA:
        assert i1["rows_pass1"] > 0 and i1["rows_pass2"] > 0
    e2 = L.ll_logdet_batched(h, dm, bounds, opts)
    i2 = h.info()
    assert np.array_equal(e1, e2)
    assert (i2["threads_pass1"], i2["threads_pass2"], i2["rows_pass1"], i2["rows_pass2"]) == \
        (i1["threads_pass1"], i1["threads_pass2"], i1["rows_pass1"], i1["rows_pass2"])
    e3 = L.ll_logdet_batched(h, dm, bounds, L.options(probes=30, seed=2, use_graph=False, step_kernel="tma"))
    assert h.info()["batch_tuned"] == 0 and h.info()["kernel_pass1"] == L.LL_KERNEL_TMA
    np.testing.assert_allclose(e3, e1, rtol=1e-12)
    for i in (0, 9):
        A, (lo, hi) = mats[i], bounds[i]
        sigma = O.sigma_of(lo)
        m = O.degree_from_bounds(lo / sigma, hi / sigma)
        want = O.logdet_leja(A, lo, hi, m, 30, 2 + i)["estimate"]
        assert abs(e1[i] - want) / abs(want) < TOL["df64"]
