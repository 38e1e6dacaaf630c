"""GPU adjoint (backward) against the oracle's frozen-basis gradient (needs a GB300).

The gradient of E(A) = n log sigma + tr(Q^T p(A~) Q) + (1/k) tr(G'^T p(A~) G') with Q, G', the
bounds, sigma and the coefficients frozen does not depend on which orthonormal basis of span(Y)
is used, so the oracle's Householder Q and the GPU's CholeskyQR2 Q give the same gradient.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from oracle import rng as ORNG
from synth import laplacian_2d, matern_2d, matern_2d_derivatives, random_spd
from tests import pins
from tests.gpu_util import TOL, lib, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


def _gpu_grad(L, h, A, lmin, lmax, degree, probes, seed, prec, kind="rademacher", ckpt=0):
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    opts = L.options(degree=degree, probes=probes, seed=seed, precision=prec, probe_kind=kind,
                     keep_for_backward=True, ckpt_stride=ckpt)
    est = L.ll_logdet_forward(h, dA, lmin, lmax, opts)
    g = L.ll_logdet_backward(h, dA, 1.0).cpu().numpy()
    return est, g, dA


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("ckpt", [0, 1, 5])
def test_backward_matches_oracle_gradient(L, h, prec, ckpt):
    A = random_spd(700, nnz_per_row=7, seed=4, empty_rows=3)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    m, probes, seed = 23, 18, 6
    _, g, _ = _gpu_grad(L, h, A, lmin, hi, m, probes, seed, prec, ckpt=ckpt)
    ref = O.logdet_leja(A, lmin, hi, m, probes, seed)
    want = O.hutchpp_grad_values(A, lmin, hi, m, ref["Q"], ref["Gp"])
    assert rel_err(g, want) < (1e-9 if prec != "f32" else 1e-4)


@pytest.mark.parametrize("prec", ["df64", "f64"])
def test_backward_gaussian_matern_theta(L, h, prec):
    """Matérn tau (kappa^2 I + L)^2 on 16 x 16 with Gaussian probes: value gradients against the
    oracle, and the kappa / tau chain through ll_param_grad against the oracle's chain."""
    torch = need_gpu()
    N, kappa, tau = 16, 0.3, 1.0
    A = matern_2d(N, kappa, tau)
    lo, hi = O.gershgorin(A)
    lmin = 0.9 * tau * (kappa * kappa + 8 * np.sin(np.pi / (2 * (N + 1))) ** 2) ** 2
    m, probes, seed = 60, 30, 2
    _, g, _ = _gpu_grad(L, h, A, lmin, hi, m, probes, seed, prec, kind="gaussian")
    ref = O.logdet_leja(A, lmin, hi, m, probes, seed, kind="gaussian")
    want = O.hutchpp_grad_values(A, lmin, hi, m, ref["Q"], ref["Gp"])
    assert rel_err(g, want) < 1e-9
    dk, dt = matern_2d_derivatives(N, kappa, tau)
    dv = torch.as_tensor(np.stack([dk, dt])).cuda()
    th = L.ll_param_grad(h, torch.as_tensor(g).cuda(), dv)
    assert th[0] == pytest.approx(float(want @ dk), rel=1e-9)
    assert th[1] == pytest.approx(float(want @ dt), rel=1e-9)


def test_backward_exact_trace_matches_closed_form(L, h):
    """k >= n: the frozen estimator is the exact polynomial trace and its parameter gradient
    approaches tr(A^-1 dA/dtheta): n / tau and 4 kappa sum 1/(kappa^2 + mu)."""
    torch = need_gpu()
    N, kappa, tau = 6, 0.3, 1.3
    A = matern_2d(N, kappa, tau)
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    lmin, lmax = 0.95 * lam[0], 1.05 * lam[-1]
    _, g, _ = _gpu_grad(L, h, A, lmin, lmax, 200, 3 * A.n, 1, "df64")
    dk, dt = matern_2d_derivatives(N, kappa, tau)
    th = L.ll_param_grad(h, torch.as_tensor(g).cuda(), torch.as_tensor(np.stack([dk, dt])).cuda())
    ex_k, ex_t = pins.dlogdet_matern_2d(N, kappa, tau)
    assert th[0] == pytest.approx(ex_k, rel=1e-5)
    assert th[1] == pytest.approx(ex_t, rel=1e-5)


def test_autograd_function(L, h):
    torch = need_gpu()
    A = laplacian_2d(30, 0.1)
    dA = L.DeviceCSR.from_host(A)
    values = dA.values.clone().requires_grad_(True)
    est = L.logdet(values, dA.rowptr, dA.colind, A.n, (0.1, 8.1), 25, 15, 3, handle=h)
    est.backward()
    ref = O.logdet_leja(A, 0.1, 8.1, 25, 15, 3)
    assert float(est.detach()) == pytest.approx(ref["estimate"], rel=1e-10)
    want = O.hutchpp_grad_values(A, 0.1, 8.1, 25, ref["Q"], ref["Gp"])
    assert rel_err(values.grad.cpu().numpy(), want) < 1e-9


def test_backward_without_forward_is_an_error(L):
    h2 = L.Handle()
    A = laplacian_2d(5, 0.1)
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_backward(h2, L.DeviceCSR.from_host(A), 1.0)
    assert ei.value.name == "LL_ERR_NO_FORWARD"


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_backward_hutchinson_matches_oracle_gradient(L, h, prec):
    """Plain Hutchinson (Eq. Léja8): the kept block is G itself (no sketch), and the adjoint's
    per-column weight is d_j / m, so the value gradients equal the oracle's frozen-probe
    gradient with an empty basis and U = G / m."""
    A = random_spd(500, nnz_per_row=6, seed=8, empty_rows=2)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    m, probes, seed = 21, 14, 3
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    opts = L.options(degree=m, probes=probes, seed=seed, precision=prec, keep_for_backward=True, estimator="hutchinson")
    est = L.ll_logdet_forward(h, dA, lmin, hi, opts)
    g = L.ll_logdet_backward(h, dA, 1.0).cpu().numpy()
    want_est = O.logdet_hutchinson(A, lmin, hi, m, probes, seed, f32=(prec == "f32"))["estimate"]
    assert abs(est - want_est) / abs(want_est) < (1e-10 if prec != "f32" else 2e-5)
    G = ORNG.probes("rademacher", seed, ORNG.STREAM_G, A.n, probes)
    want = O.hutchpp_grad_values(A, lmin, hi, m, np.zeros((A.n, 0)), G)
    assert rel_err(g, want) < (1e-9 if prec != "f32" else 1e-4)
    with pytest.raises(L.LejaError) as ei:
        L.ll_kept_basis(h)
    assert ei.value.name == "LL_ERR_UNSUPPORTED"


# --------------------------------------------------- derivative through the sketch's QR

@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_backward_qr_matches_oracle_full_gradient(L, h, prec):
    """ll_logdet_backward_qr against the oracle's frozen-basis gradient plus the term through
    Q = orth(p(A~) S) (same S and G: streams 0 and 1 of the seed)."""
    A = random_spd(700, nnz_per_row=7, seed=4, empty_rows=3)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    m, probes, seed = 23, 18, 6
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    L.ll_logdet_forward(h, dA, lmin, hi, L.options(degree=m, probes=probes, seed=seed, precision=prec,
                                                    keep_for_backward=True))
    g = L.ll_logdet_backward(h, dA, 1.0, through_qr=True).cpu().numpy()
    S, G = O.make_probes(A.n, probes // 3, seed)
    want = O.hutchpp_full_grad_values(A, lmin, hi, m, S, G)
    assert rel_err(g, want) < (1e-9 if prec != "f32" else 1e-4)
    frozen = L.ll_logdet_backward(h, dA, 1.0).cpu().numpy()
    assert rel_err(frozen, want) > 1e-3   # the QR term is not negligible here


def test_backward_qr_is_the_frozen_gradient_without_a_qr(L, h):
    """Hutchinson (no sketch) and k >= n (Q spans R^n, Gamma = 0): both backwards agree."""
    A = random_spd(300, seed=2)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    dA = L.DeviceCSR.from_host(A)
    L.ll_logdet_forward(h, dA, lmin, hi, L.options(degree=20, probes=7, seed=1, estimator="hutchinson",
                                                    keep_for_backward=True))
    assert L.ll_logdet_backward(h, dA, 2.0, through_qr=True).equal(L.ll_logdet_backward(h, dA, 2.0))
    B = random_spd(12, seed=5)
    lo, hi = O.gershgorin(B)
    dB = L.DeviceCSR.from_host(B)
    L.ll_logdet_forward(h, dB, max(lo, 0.05), hi, L.options(degree=20, probes=36, seed=1, keep_for_backward=True))
    assert L.ll_logdet_backward(h, dB, 1.0, through_qr=True).equal(L.ll_logdet_backward(h, dB, 1.0))


@pytest.mark.parametrize("prec", ["df64", "f64"])
def test_backward_qr_theta_chain_matches_finite_differences_of_the_gpu_estimate(L, h, prec):
    """GMRF Q(theta) = I + theta Adj on 30 x 30: d/dtheta of the GPU estimate (same probes, fixed
    bounds and degree; Q and G' recomputed) by central differences, against the through-QR
    gradient chained to theta."""
    torch = need_gpu()
    from synth import gmrf_theta
    theta, eps = -0.2, 1e-5
    A = gmrf_theta(30, theta)
    lo, hi = 1 - 4 * 0.21, 1 + 4 * 0.21
    opts = L.options(degree=40, probes=24, seed=3, precision=prec, keep_for_backward=True)
    est = {}
    for t in (theta - eps, theta + eps):
        dA = L.DeviceCSR.from_host(gmrf_theta(30, t))
        est[t] = L.ll_logdet_forward(h, dA, lo, hi, opts)
    fd = (est[theta + eps] - est[theta - eps]) / (2 * eps)
    dA = L.DeviceCSR.from_host(A)
    L.ll_logdet_forward(h, dA, lo, hi, opts)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    dv = torch.as_tensor((A.colind != rows).astype(np.float64)).cuda()
    full = L.ll_param_grad(h, L.ll_logdet_backward(h, dA, 1.0, through_qr=True), dv)[0]
    frozen = L.ll_param_grad(h, L.ll_logdet_backward(h, dA, 1.0), dv)[0]
    assert full == pytest.approx(fd, rel=1e-6)
    assert abs(frozen - fd) > 100 * abs(full - fd)


def test_autograd_through_qr(L, h):
    torch = need_gpu()
    A = random_spd(500, seed=8)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    dA = L.DeviceCSR.from_host(A)
    vals = dA.values.clone().requires_grad_(True)
    est = L.logdet(vals, dA.rowptr, dA.colind, A.n, (lmin, hi), 25, 15, seed=2, handle=h, through_qr=True)
    est.backward()
    S, G = O.make_probes(A.n, 5, 2)
    want = O.hutchpp_full_grad_values(A, lmin, hi, 25, S, G)
    assert rel_err(vals.grad.cpu().numpy(), want) < 1e-9


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_backward_from_kept_w_equals_recomputed(L, h, prec):
    """By default both passes keep W_1 .. W_m for the backward (ll_info.kept_w_steps and
    kept_w_steps_pass1 = m); under an explicit checkpoint stride the backward recomputes them.
    The through-QR term's F [Q | G'] then comes from the kept W_j (a weighted sum) instead of a
    P-axpy sweep, with the same numbers. The W_j are the
    same numbers either way, so the two gradients are identical, and a through-QR backward in
    between (its own checkpoints) leaves the kept ones intact."""
    A = random_spd(900, nnz_per_row=6, seed=11, empty_rows=2)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    m = 17
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    grads = {}
    for ckpt in (0, 4):
        L.ll_logdet_forward(h, dA, lmin, hi, L.options(degree=m, probes=21, seed=5, precision=prec,
                                                        keep_for_backward=True, ckpt_stride=ckpt))
        info = h.info()
        assert info["kept_w_steps"] == (m if ckpt == 0 else 0)
        assert info["kept_w_steps_pass1"] == (m if ckpt == 0 else 0)
        g = L.ll_logdet_backward(h, dA, 1.0)
        gq = L.ll_logdet_backward(h, dA, 1.0, through_qr=True)
        assert L.ll_logdet_backward(h, dA, 1.0).equal(g)
        grads[ckpt] = (g, gq)
    assert grads[0][0].equal(grads[4][0])
    assert grads[0][1].equal(grads[4][1])
    ref = O.logdet_leja(A, lmin, hi, m, 21, 5)
    want = O.hutchpp_grad_values(A, lmin, hi, m, ref["Q"], ref["Gp"])
    assert rel_err(grads[0][0].cpu().numpy(), want) < (1e-9 if prec != "f32" else 1e-4)


def test_backward_from_kept_w_on_a_banded_matrix(L, h):
    """A banded matrix: when its trace pass keeps the W_j it runs on the one-step kernels (the
    multi-step kernel keeps only every fourth W_j in memory); pass 1 stays banded. Same gradient
    as the checkpointed backward after a banded trace pass."""
    from synth import pentadiagonal
    A = pentadiagonal(1500, seed=3)
    lo, hi = O.gershgorin(A)
    dA = L.DeviceCSR.from_host(A)
    out = {}
    for ckpt in (0, 3):
        L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=11, probes=15, seed=2, keep_for_backward=True,
                                                      ckpt_stride=ckpt))
        info = h.info()
        assert info["kernel_pass1"] == L.LL_KERNEL_BAND and info["kept_w_steps_pass1"] == 0
        assert (info["kernel_pass2"] == L.LL_KERNEL_BAND) == (ckpt != 0)
        out[ckpt] = L.ll_logdet_backward(h, dA, 1.0)
    assert out[0].equal(out[3])


@pytest.mark.parametrize("prec", ["df64", "f32"])
def test_backward_from_forward_written_checkpoints(L, h, prec):
    """A keep budget too small for every W_j but large enough for the checkpoints at stride 3
    (5.5 blocks: stride 2 needs 8, stride 3 needs ceil(17/3) - 1 = 5): the trace pass writes W_3,
    W_6, ..., W_15 for the backward, which then recomputes only inside segments. Both gradients
    are bit-identical to an explicit ckpt_stride = 3 (the backward checkpoints itself), and the
    kept checkpoints survive a first backward. Under a budget below the largest stride's 3
    blocks nothing is kept and the result is the same."""
    A = random_spd(900, nnz_per_row=6, seed=11, empty_rows=2)
    lo, hi = O.gershgorin(A)
    lmin = max(lo, 0.05)
    m, probes = 17, 21
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    l2 = 16 if prec == "f32" else 14                      # [Q | G'] block: 14 columns (FP32: 16)
    blk = A.n * l2 * (4 if prec == "f32" else 8)
    out = {}
    try:
        for name, budget, ckpt in (("fwd", int(5.5 * blk), 0), ("bwd", 0, 3), ("none", int(2.5 * blk), 0)):
            h.set_keep_budget(budget)
            L.ll_logdet_forward(h, dA, lmin, hi, L.options(degree=m, probes=probes, seed=5, precision=prec,
                                                            keep_for_backward=True, ckpt_stride=ckpt))
            info = h.info()
            want_stride, want_steps = {"fwd": (3, 5), "bwd": (0, 0), "none": (0, 0)}[name]
            assert (info["kept_w_stride"], info["kept_w_steps"]) == (want_stride, want_steps)
            g1 = L.ll_logdet_backward(h, dA, 1.0)
            gq = L.ll_logdet_backward(h, dA, 1.0, through_qr=True)
            g2 = L.ll_logdet_backward(h, dA, 1.0)
            assert g1.equal(g2)
            out[name] = (g1, gq)
    finally:
        h.set_keep_budget(0)
    for name in ("bwd", "none"):
        assert out["fwd"][0].equal(out[name][0])
        assert out["fwd"][1].equal(out[name][1])
    ref = O.logdet_leja(A, lmin, hi, m, probes, 5)
    want = O.hutchpp_grad_values(A, lmin, hi, m, ref["Q"], ref["Gp"])
    assert rel_err(out["fwd"][0].cpu().numpy(), want) < (1e-9 if prec != "f32" else 1e-4)


def test_backward_rejects_a_nonsymmetric_matrix(L, h):
    """The reverse recurrence uses B^T = B: a stored (r, c) whose (c, r) partner differs fails."""
    A = random_spd(400, seed=3)
    lo, hi = O.gershgorin(A)
    vals = np.array(A.values, dtype=np.float64)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    e = int(np.nonzero(np.asarray(A.colind) != rows)[0][0])
    dA = L.DeviceCSR.from_host(A)
    L.ll_logdet_forward(h, dA, max(lo, 0.05), hi, L.options(degree=10, probes=6, seed=1, keep_for_backward=True))
    assert L.ll_logdet_backward(h, dA, 1.0).shape[0] == A.nnz
    vals[e] *= 1.5
    dA.values.copy_(need_gpu().as_tensor(vals))
    with pytest.raises(L.LejaError) as ei:
        L.ll_logdet_backward(h, dA, 1.0)
    assert ei.value.name == "LL_ERR_INVALID_ARG"


def test_autograd_refuses_a_stale_forward(L):
    """The handle keeps only its last forward: differentiating an earlier estimate on the same
    handle is refused, not answered with the later forward's gradient."""
    torch = need_gpu()
    h2 = L.Handle()
    A, B = laplacian_2d(20, 0.1), laplacian_2d(20, 0.2)
    dA, dB = L.DeviceCSR.from_host(A), L.DeviceCSR.from_host(B)
    va = dA.values.clone().requires_grad_(True)
    vb = dB.values.clone().requires_grad_(True)
    ea = L.logdet(va, dA.rowptr, dA.colind, A.n, (0.1, 8.1), 20, 6, 1, handle=h2)
    eb = L.logdet(vb, dB.rowptr, dB.colind, B.n, (0.2, 8.2), 20, 6, 1, handle=h2)
    eb.backward()
    assert vb.grad is not None
    with pytest.raises(L.LejaError) as ei:
        ea.backward()
    assert ei.value.name == "LL_ERR_NO_FORWARD"
    with pytest.raises(L.LejaError):
        h2.set_keep_budget(-1)
    del torch


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("mat", ["matern", "irregular"])
def test_fused_and_separate_contraction_agree_with_the_oracle(L, prec, mat):
    """The reverse step with the gradient contraction fused in (ll_set_adjoint_fusion "on") and
    the reverse step followed by the separate contraction ("off"), both on the TMA step kernel
    with one column pair per thread: each against the oracle's frozen-basis gradient, and the two
    against each other to rounding (each entry's column pairs are summed in another order)."""
    if mat == "matern":
        A = matern_2d(40, 0.3, 1.0)
        lmin = 0.0081
    else:
        A = random_spd(900, nnz_per_row=9, seed=7, empty_rows=4)
        lmin = max(O.gershgorin(A)[0], 0.05)
    hi = O.gershgorin(A)[1]
    m, probes, seed = 20, 30, 3
    got = {}
    for mode in ("on", "off"):
        hh = L.Handle()
        hh.set_step_config("tma", 0, 1)
        hh.set_adjoint_fusion(mode)
        _, got[mode], _ = _gpu_grad(L, hh, A, lmin, hi, m, probes, seed, prec)
        assert hh.info()["adjoint_fused"] == (1 if mode == "on" else 0)
    ref = O.logdet_leja(A, lmin, hi, m, probes, seed)
    want = O.hutchpp_grad_values(A, lmin, hi, m, ref["Q"], ref["Gp"])
    for mode in ("on", "off"):
        assert rel_err(got[mode], want) < (1e-9 if prec != "f32" else 1e-4)
    assert np.max(np.abs(got["on"] - got["off"])) <= 1e-12 * np.max(np.abs(got["off"]))


def test_adjoint_fusion_mode_is_checked(L):
    hh = L.Handle()
    with pytest.raises(L.LejaError) as ei:
        hh.check(hh._lib.ll_set_adjoint_fusion(hh.ptr, 7))
    assert ei.value.name == "LL_ERR_INVALID_ARG"
