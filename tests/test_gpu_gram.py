"""CholeskyQR2's Gram products on the tensor cores against FP64 references (needs a GB300).

The tensor-core kernel writes every column in fixed point per batch of 512 rows as six 8-bit digit
slices, multiplies the slices exactly in FP32 accumulators and sums the scaled products in
double-float: about 47 bits below each column's batch maximum, the accuracy of the double-float
kernel it replaces. Both are checked against a float64 product of the same (rounded) inputs, with a
norm-wise bound |G_jl - ref_jl| <= tol ||x_j|| ||z_l|| (the float64 product's own error is about
n 2^-53 of that in the worst case), over ragged row counts (partial batches and chunks), the widths
at the edges of the tile layout (1, 10, 21, 22, 33, 40), columns of very different scales, zero
columns and both operand layouts. Widths above 36 carry six digits (42 bits), so their bound is
1e-12 instead of 1e-13.
"""
from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_util import lib, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


@pytest.fixture(scope="module")
def h(L):
    return L.Handle()


def _ref(X, Z):
    return X.T @ Z


def _bound(X, Z):
    return np.outer(np.linalg.norm(X, axis=0), np.linalg.norm(Z, axis=0))


def _tol(method, k):
    # seven 7-bit digits up to width 36 (49 bits), six above (42 bits: about 2.3e-13)
    return 1e-12 if method == "tensor" and k > 36 else 1e-13


def _cols(n, k, seed, scales=None):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k))
    if scales is not None:
        X *= np.asarray(scales)[None, :]
    return X


@pytest.mark.parametrize("k", [1, 10, 21, 22, 33, 40])
@pytest.mark.parametrize("n", [100, 511, 1025, 100_003])
def test_symmetric_gram_df64_layout(L, h, k, n):
    torch = need_gpu()
    X = _cols(n, k, seed=k + n)
    B = L.df64_block(X)
    # the reference takes the double-float values the block holds
    hi = B.reshape(n, -1, 4)
    xr = np.zeros((n, B.shape[1] // 2))
    xr[:, 0::2] = hi[:, :, 0].astype(np.float64) + hi[:, :, 2].astype(np.float64)
    xr[:, 1::2] = hi[:, :, 1].astype(np.float64) + hi[:, :, 3].astype(np.float64)
    xr = xr[:, :k]
    dX = torch.as_tensor(B).cuda()
    want = _ref(xr, xr)
    bound = _bound(xr, xr)
    for method in ("tensor", "dfloat"):
        got = L.ll_gram(h, dX, None, method=method, kx=k).cpu().numpy()
        assert np.all(np.abs(got - want) <= _tol(method, k) * bound), method
        assert np.array_equal(got, got.T)


@pytest.mark.parametrize("kx,kz", [(33, 33), (10, 10), (40, 40), (20, 20), (7, 3)])
def test_cross_gram_f64(L, h, kx, kz):
    """X^T Z with FP64 operands (Q^T G of step 6 and the through-QR adjoint's products)."""
    torch = need_gpu()
    n = 70_001
    X = _cols(n, kx, seed=1)
    Z = np.sign(_cols(n, kz, seed=2))           # Rademacher-like
    dX, dZ = torch.as_tensor(X).cuda(), torch.as_tensor(Z).cuda()
    want, bound = _ref(X, Z), _bound(X, Z)
    for method in ("tensor", "dfloat"):
        got = L.ll_gram(h, dX, dZ, method=method).cpu().numpy()
        assert np.all(np.abs(got - want) <= _tol(method, max(kx, kz)) * bound), method


def test_gram_scales_zero_columns_and_strided_operands(L, h):
    """Columns from 1e-9 to 1e9 and an all-zero column (each column has its own fixed-point scale),
    rows of zeros, a leading dimension wider than the block, and a tail of 3 rows."""
    torch = need_gpu()
    n, k = 4 * 512 + 3, 12
    scales = np.logspace(-9, 9, k)
    scales[5] = 0.0
    X = _cols(n, k, seed=9, scales=scales)
    X[100:700] = 0.0
    W = np.zeros((n, k + 5))
    W[:, :k] = X
    dW = torch.as_tensor(W).cuda()[:, :k]
    want, bound = _ref(X, X), _bound(X, X)
    got = L.ll_gram(h, dW, None, method="tensor").cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-13 * bound + 1e-300)
    assert np.all(got[5] == 0.0) and np.all(got[:, 5] == 0.0)
    Z = _cols(n, 3, seed=4)
    got = L.ll_gram(h, dW, torch.as_tensor(Z).cuda(), method="tensor").cpu().numpy()
    assert np.all(np.abs(got - _ref(X, Z)) <= 1e-13 * _bound(X, Z) + 1e-300)


def test_gram_tensor_width_limit(L, h):
    torch = need_gpu()
    X = torch.as_tensor(_cols(1000, 43, seed=3)).cuda()
    with pytest.raises(L.LejaError) as ei:
        L.ll_gram(h, X, None, method="tensor")
    assert ei.value.name == "LL_ERR_UNSUPPORTED"
    got = L.ll_gram(h, X, None, method="auto").cpu().numpy()   # falls back to the double-float kernel
    Xh = X.cpu().numpy()
    assert np.all(np.abs(got - Xh.T @ Xh) <= 1e-13 * _bound(Xh, Xh))


@pytest.mark.parametrize("prec", ["df64", "f64", "f32"])
def test_forward_with_either_gram_kernel(L, h, prec):
    """The estimator's CholeskyQR2 with the tensor-core Grams and with the double-float ones: the
    estimates agree to rounding, and both match the oracle on the same probes."""
    from oracle import logdet as O
    from synth import laplacian_3d
    from tests.gpu_util import TOL
    A = laplacian_3d(30, 0.05)
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    est = {}
    for g in ("tensor", "dfloat"):
        est[g] = L.ll_logdet_forward(h, dA, 0.05, 12.05, L.options(degree=20, probes=99, seed=4, precision=prec, qr_gram=g))
    assert abs(est["tensor"] - est["dfloat"]) <= 1e-12 * abs(est["dfloat"])
    want = O.logdet_leja(A, 0.05, 12.05, 20, 99, 4, f32=(prec == "f32"))["estimate"]
    assert abs(est["tensor"] - want) <= TOL[prec] * abs(want)


@pytest.mark.parametrize("layout", ["df64", "f64"])
def test_gram_many_exact_batches_per_cta(L, h, layout):
    """More than 4096 rows per CTA (the exact FP32 sums are drained into the double-float sums
    several times), with a ragged last chunk."""
    torch = need_gpu()
    n, k = 152 * 4096 * 2 + 4097, 33
    X = _cols(n, k, seed=21)
    if layout == "df64":
        B = L.df64_block(X)
        hi = B.reshape(n, -1, 4)
        xr = np.zeros((n, B.shape[1] // 2))
        xr[:, 0::2] = hi[:, :, 0].astype(np.float64) + hi[:, :, 2].astype(np.float64)
        xr[:, 1::2] = hi[:, :, 1].astype(np.float64) + hi[:, :, 3].astype(np.float64)
        X, dX = xr[:, :k], torch.as_tensor(B).cuda()
    else:
        dX = torch.as_tensor(X).cuda()
    got = L.ll_gram(h, dX, None, method="tensor", kx=k).cpu().numpy()
    assert np.all(np.abs(got - X.T @ X) <= 1e-13 * _bound(X, X))
    Z = np.sign(_cols(n, 20, seed=22))
    got = L.ll_gram(h, torch.as_tensor(X).cuda(), torch.as_tensor(Z).cuda(), method="tensor").cpu().numpy()
    assert np.all(np.abs(got - X.T @ Z) <= 1e-13 * _bound(X, Z))


@pytest.mark.parametrize("k", [10, 33])
def test_auto_gram_is_one_of_the_kernels_and_repeats(L, k):
    """LL_GRAM_AUTO times both kernels on the first product of a shape and keeps the faster: the
    first and later results are bit-identical, and equal to one of the two kernels' results."""
    torch = need_gpu()
    h2 = L.Handle()
    X = torch.as_tensor(_cols(200_003, k, seed=k)).cuda()
    first = L.ll_gram(h2, X, None, method="auto").cpu().numpy()
    again = L.ll_gram(h2, X, None, method="auto").cpu().numpy()
    assert np.array_equal(first, again)
    tc = L.ll_gram(h2, X, None, method="tensor").cpu().numpy()
    df = L.ll_gram(h2, X, None, method="dfloat").cpu().numpy()
    assert np.array_equal(first, tc) or np.array_equal(first, df)
