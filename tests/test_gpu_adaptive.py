"""Algorithm 2's stopping rule on the GPU against the oracle (needs a GB300 and the library).

The rule |d_m| ||w_m||_2 <= tol turns a floating-point norm into an integer degree per column.
Each case picks its tolerance where the oracle's degrees do not change under a relative
perturbation of it (1e-8 for the FP64-class paths, 1e-3 for FP32-mixed), so that the GPU's
norms, summed in another order, must take the same decisions. The degrees are then compared
exactly, the blocks and estimates at the parity bar.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from synth import diagonal, laplacian_2d, random_spd
from tests.gpu_util import TOL, lib, need_gpu, rel_err

pytestmark = pytest.mark.gpu

MARGIN = {"f64": 1e-8, "df64": 1e-8, "f32": 1e-3}


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


def _robust_tol(decide, tol0, margin):
    """The first of tol0 * 1.37^i whose decisions are the same at tol (1 - margin) and tol (1 + margin)."""
    tol = tol0
    for _ in range(40):
        a, b = decide(tol * (1 - margin)), decide(tol * (1 + margin))
        if all(np.array_equal(x, y) for x, y in zip(a, b)):
            return tol
        tol *= 1.37
    raise AssertionError("no tolerance clear of the decision boundaries")


def _apply_oracle(A, lmin, lmax, degree, V, tol, f32):
    xi, c, g, d, _ = O.newton_leja_setup(lmin, lmax, degree)
    return O.leja_apply_columns_adaptive(O._scipy(A), V, xi, d, c, g, tol, 1.0, f32)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("kernel", ["gather", "tma"])
@pytest.mark.parametrize("b", [1, 5, 12])
def test_apply_poly_tol_matches_oracle(L, h, prec, kernel, b):
    """Columns of different scales stop at different degrees; odd widths have a pad column."""
    torch = need_gpu()
    A = laplacian_2d(43, 0.3)                     # n = 1849: several tiles and a ragged tail
    lmin, lmax, degree = 0.3, 8.3, 60
    rs = np.random.default_rng(b)
    V = rs.standard_normal((A.n, b)) * np.logspace(-3, 3, b)[None, :]
    f32 = prec == "f32"
    tol = _robust_tol(lambda t: [_apply_oracle(A, lmin, lmax, degree, V, t, f32)[1]], 1e-7, MARGIN[prec])
    want, wdeg = _apply_oracle(A, lmin, lmax, degree, V, tol, f32)
    assert b == 1 or len(set(wdeg.tolist())) > 1
    assert 0 < wdeg.min() < degree
    dA = L.DeviceCSR.from_host(A, "f32" if f32 else "f64")
    h.set_step_config(kernel, 0, 0)
    try:
        got, gdeg = L.ll_apply_poly_tol(h, dA, lmin, lmax, degree, tol, torch.as_tensor(V).cuda(), prec)
    finally:
        h.set_step_config("auto", 0, 0)
    assert gdeg.tolist() == wdeg.tolist()
    assert rel_err(got.cpu().numpy(), want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_apply_poly_tol_degree_cap_and_immediate_stop(L, h, prec):
    """A tolerance below every term runs to the cap and equals the fixed-degree block; one
    above |d_0| ||v|| stops every column at degree 0 (PV = d_0 V)."""
    torch = need_gpu()
    A = random_spd(1500, seed=4, empty_rows=3, dense_row=True)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    V = np.random.default_rng(1).standard_normal((A.n, 6))
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    Vd = torch.as_tensor(V).cuda()
    got, deg = L.ll_apply_poly_tol(h, dA, lmin, hi, 30, 1e-300, Vd, prec)
    fixed = L.ll_apply_poly(h, dA, lmin, hi, 30, Vd, prec)
    assert deg.tolist() == [30] * 6
    assert torch.equal(got, fixed)
    got, deg = L.ll_apply_poly_tol(h, dA, lmin, hi, 30, 1e300, Vd, prec)
    d0 = O.newton_leja_setup(lmin, hi, 30)[3][0]
    assert deg.tolist() == [0] * 6
    assert rel_err(got.cpu().numpy(), d0 * V) < TOL[prec]


def _fwd_oracle(A, lmin, lmax, degree, probes, seed, prec, tol, est, kind="rademacher"):
    f32 = prec == "f32"
    if est == "hutchinson":
        r = O.logdet_hutchinson(A, lmin, lmax, degree, probes, seed, kind=kind, f32=f32, tol=tol)
        return r, [np.zeros(0, dtype=np.int64), r["deg_g"]]
    r = O.logdet_leja(A, lmin, lmax, degree, probes, seed, kind=kind, f32=f32, tol=tol)
    return r, [r["deg_s"], np.concatenate([r["deg_q"], r["deg_g"]])]


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("est,kind", [("hutchpp", "rademacher"), ("hutchpp", "gaussian"), ("hutchinson", "gaussian")])
def test_forward_tol_matches_oracle(L, h, prec, est, kind):
    """Both passes under the rule: per-column final degrees (the sketch columns; then [Q | G'],
    or the Hutchinson probes) equal the oracle's, and the estimate is at the parity bar."""
    A = laplacian_2d(36, 0.5)
    lmin, hi, degree, probes = 0.5, 8.5, 80, 15
    tol = _robust_tol(lambda t: _fwd_oracle(A, lmin, hi, degree, probes, 3, prec, t, est, kind)[1], 1e-5, MARGIN[prec])
    r, (want1, want2) = _fwd_oracle(A, lmin, hi, degree, probes, 3, prec, tol, est, kind)
    assert want2.max() < degree
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    opts = L.options(degree=degree, probes=probes, seed=3, precision=prec, estimator=est, probe_kind=kind, tol=tol)
    got = L.ll_logdet_forward(h, dA, lmin, hi, opts)
    info = h.info()
    assert L.ll_stop_degrees(h, 1).tolist() == want1.tolist()
    assert L.ll_stop_degrees(h, 2).tolist() == want2.tolist()
    assert info["deg_max_pass2"] == int(want2.max())
    assert info["deg_mean_pass2"] == pytest.approx(float(np.mean(want2)))
    assert abs(got - r["estimate"]) / abs(r["estimate"]) < TOL[prec]
    # the graph replay of the same call takes the same decisions
    again = L.ll_logdet_forward(h, dA, lmin, hi, opts)
    assert again == got
    assert L.ll_stop_degrees(h, 2).tolist() == want2.tolist()


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_forward_tiny_tol_is_the_fixed_degree(L, h, prec):
    """tol below every term: the same estimate as tol = 0, every column at the degree."""
    A = laplacian_2d(60, 0.2)
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    fixed = L.ll_logdet_forward(h, dA, 0.2, 8.2, L.options(degree=40, probes=21, seed=5, precision=prec))
    assert L.ll_stop_degrees(h, 2).tolist() == [40] * 14
    got = L.ll_logdet_forward(h, dA, 0.2, 8.2, L.options(degree=40, probes=21, seed=5, precision=prec, tol=1e-300))
    assert L.ll_stop_degrees(h, 1).tolist() == [40] * 7
    assert L.ll_stop_degrees(h, 2).tolist() == [40] * 14
    assert abs(got - fixed) <= 1e-14 * abs(fixed)


def test_forward_tol_rademacher_diagonal_closed_form(L, h):
    """Rademacher Hutchinson on a diagonal matrix: every probe has the same term norms, so every
    column stops at the same degree, and the estimate equals the oracle's exact polynomial trace
    at that degree."""
    dvals = np.linspace(0.2, 6.0, 4000)
    A = diagonal(dvals)
    tol = _robust_tol(lambda t: _fwd_oracle(A, 0.2, 6.0, 70, 4, 3, "df64", t, "hutchinson")[1], 1e-6, 1e-8)
    r, (_, want2) = _fwd_oracle(A, 0.2, 6.0, 70, 4, 3, "df64", tol, "hutchinson")
    assert len(set(want2.tolist())) == 1
    dA = L.DeviceCSR.from_host(A)
    got = L.ll_logdet_forward(h, dA, 0.2, 6.0, L.options(degree=70, probes=4, seed=3, estimator="hutchinson", tol=tol))
    assert L.ll_stop_degrees(h, 2).tolist() == want2.tolist()
    assert got == pytest.approx(r["estimate"], rel=1e-12)


def test_tol_argument_errors(L, h):
    torch = need_gpu()
    A = laplacian_2d(20, 0.5)
    dA = L.DeviceCSR.from_host(A)
    for opts, code in ((L.options(tol=-1.0), "LL_ERR_INVALID_ARG"), (L.options(tol=float("nan")), "LL_ERR_INVALID_ARG"),
                       (L.options(tol=1e-3, keep_for_backward=True), "LL_ERR_UNSUPPORTED")):
        with pytest.raises(L.LejaError) as ei:
            L.ll_logdet_forward(h, dA, 0.5, 8.5, opts)
        assert ei.value.name == code
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_batched(h, [dA], [(0.5, 8.5)], L.options(probes=30, tol=1e-3))
    assert ei.value.name == "LL_ERR_UNSUPPORTED"
    with pytest.raises(L.LejaError) as ei:
        L.ll_apply_poly_tol(h, dA, 0.5, 8.5, 20, 0.0, torch.ones((A.n, 2), dtype=torch.float64).cuda())
    assert ei.value.name == "LL_ERR_INVALID_ARG"
    with pytest.raises(L.LejaError) as ei:
        L.ll_stop_degrees(h, 3)
    assert ei.value.name == "LL_ERR_INVALID_ARG"
