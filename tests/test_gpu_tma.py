"""The TMA-fed step kernel (tile::gather4 into a shared-memory pipeline) against the
register-gather kernel and the oracle (needs a GB300).

Both kernels run the same per-row arithmetic in the same entry order, so p(A)V (pass 1: the
P-axpy), the adjoint's W_j and Lambda_j, and hence the value gradients agree bit for bit; the
pass-2 traces are sums over CTAs whose count differs between the kernels, so estimates agree to
rounding. Cases cover ragged last tiles, odd widths (the pad column of a pair), widths of one and
two, tiles whose entries exceed the gather capacity (power-law rows read directly), rows without
entries besides the diagonal, a dense row, and both CTA shapes (one 512-thread CTA per SM, two of
256).
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import logdet as O
from oracle import rng as R
from synth import laplacian_3d, matern_2d, powerlaw_laplacian, random_spd
from tests.gpu_util import TOL, lib, need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    return lib()


def _apply(L, A, lo, hi, m, V, prec, kernel, threads=0, rpt=0):
    torch = need_gpu()
    h = L.Handle()
    h.set_step_config(kernel, threads, rpt)
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    out = L.ll_apply_poly(h, dA, lo, hi, m, torch.as_tensor(V).cuda(), prec).cpu().numpy()
    return out, h.info()


MATS = {
    "lap3d_24": lambda: (laplacian_3d(24, 0.05), 0.05, 12.05),
    "matern_60": lambda: (matern_2d(60, 0.3, 1.0), 0.0081, 65.4481),
    "powerlaw_4096": lambda: (powerlaw_laplacian(1 << 12, seed=3), 0.01, None),
    "spd_irregular": lambda: (random_spd(777, 6, seed=5, empty_rows=9, dense_row=True), None, None),
}


def _mat(name):
    A, lo, hi = MATS[name]()
    if lo is None or hi is None:
        glo, ghi = O.gershgorin(A)
        lo = lo if lo is not None else max(glo, 1e-3)
        hi = hi if hi is not None else ghi
    return A, lo, hi


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("b", [1, 2, 7, 33, 66])
def test_tma_matches_gather_bitwise_and_oracle(L, name, prec, b):
    A, lo, hi = _mat(name)
    m = 12
    V = R.rademacher(7, R.STREAM_S, A.n, b)
    g, ig = _apply(L, A, lo, hi, m, V, prec, "gather")
    t, it = _apply(L, A, lo, hi, m, V, prec, "tma")
    assert ig["kernel_pass1"] == L.LL_KERNEL_GATHER
    assert it["kernel_pass1"] == L.LL_KERNEL_TMA
    assert np.array_equal(g, t)
    want = O.apply_poly(A, V[:, : min(b, 3)], lo, hi, m, f32=(prec == "f32"))
    assert rel_err(t[:, : min(b, 3)], want) < TOL[prec]


@pytest.mark.parametrize("prec", ["df64", "f32"])
def test_tma_two_ctas_per_sm_matches(L, prec):
    A, lo, hi = _mat("lap3d_24")
    V = R.rademacher(3, R.STREAM_S, A.n, 66)
    g, _ = _apply(L, A, lo, hi, 9, V, prec, "gather")
    t, it = _apply(L, A, lo, hi, 9, V, prec, "tma", threads=256)
    assert it["kernel_pass1"] == L.LL_KERNEL_TMA and it["threads_pass1"] <= 256 + 96  # consumers + producer warps
    assert np.array_equal(g, t)


def test_tma_long_rows_beyond_gather_capacity(L):
    """A tile with one row of 3000 entries: everything past the gather capacity is read directly."""
    n = 2048
    rng = np.random.default_rng(1)
    M = np.zeros((n, n))
    hub = 1000
    nb = rng.choice(n, 3000 if n > 3000 else n - 1, replace=False)
    nb = nb[nb != hub]
    M[hub, nb] = -rng.uniform(0.5, 1.5, nb.size)
    M[nb, hub] = M[hub, nb]
    for i in range(n):
        j = (i + 1) % n
        M[i, j] = M[j, i] = -0.5
    np.fill_diagonal(M, 0.0)
    np.fill_diagonal(M, -M.sum(axis=1) + 0.05)
    from synth import csr_from_dense
    A = csr_from_dense(M)
    lo, hi = 0.05, O.gershgorin(A)[1]
    V = R.rademacher(5, R.STREAM_S, n, 20)
    for prec in ("df64", "f32"):
        g, _ = _apply(L, A, lo, hi, 10, V, prec, "gather")
        t, it = _apply(L, A, lo, hi, 10, V, prec, "tma")
        assert it["kernel_pass1"] == L.LL_KERNEL_TMA
        assert np.array_equal(g, t)
        want = O.apply_poly(A, V[:, :2], lo, hi, 10, f32=(prec == "f32"))
        assert rel_err(t[:, :2], want) < TOL[prec]


def _six_band_matrix(n: int = 4096, seed: int = 8):
    """Symmetric, diagonally dominant: the ±1 neighbours, six far bands (offsets ±64, ±128, ±192,
    every far entry on a diagonal run) and a few isolated far pairs. Validation counts the runs,
    so a tile's gather rows cover four extra windows; the other two bands' entries and the isolated
    ones then go past the gather capacity and are read directly."""
    import scipy.sparse as sp
    from synth import CSR
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for off in (1, 64, 128, 192):
        i = np.arange(n - off)
        rows += [i, i + off]
        cols += [i + off, i]
    iso_r = rng.integers(0, n, 40)
    iso_c = (iso_r + rng.integers(600, n - 600, 40)) % n
    keep = np.abs(iso_r - iso_c) > 200
    rows += [iso_r[keep], iso_c[keep]]
    cols += [iso_c[keep], iso_r[keep]]
    r, c = np.concatenate(rows), np.concatenate(cols)
    v = -rng.uniform(0.2, 1.0, r.size)
    M = sp.coo_matrix((v, (r, c)), shape=(n, n)).tocsr()
    M.sum_duplicates()
    M = (M + M.T) * 0.5
    d = -np.asarray(M.sum(axis=1)).ravel() + 0.05
    M = (M + sp.diags(d)).tocsr()
    M.sort_indices()
    return CSR.from_scipy(M)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
@pytest.mark.parametrize("b", [7, 66])
def test_tma_windows_and_gathers_past_the_run_capacity(L, prec, b):
    """Far entries on runs size the gather rows for four extra windows: the bands beyond them and
    the isolated far entries overflow into direct loads, bit for bit as the register kernel."""
    A = _six_band_matrix()
    lo, hi = 0.05, O.gershgorin(A)[1]
    V = R.rademacher(11, R.STREAM_S, A.n, b)
    g, _ = _apply(L, A, lo, hi, 8, V, prec, "gather")
    t, it = _apply(L, A, lo, hi, 8, V, prec, "tma")
    assert it["kernel_pass1"] == L.LL_KERNEL_TMA
    assert np.array_equal(g, t)
    want = O.apply_poly(A, V[:, :3], lo, hi, 8, f32=(prec == "f32"))
    assert rel_err(t[:, :3], want) < TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_tma_forward_and_backward(L, prec):
    """Forward (pass 1 and the trace pass) and the adjoint (recompute and reverse steps)."""
    torch = need_gpu()
    A, lo, hi = _mat("lap3d_24")
    dA = L.DeviceCSR.from_host(A, "f32" if prec == "f32" else "f64")
    res = {}
    for kernel in ("gather", "tma"):
        h = L.Handle()
        h.set_step_config(kernel, 0, 0)
        est = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=20, probes=30, seed=4, precision=prec,
                                                              keep_for_backward=True, step_kernel=kernel))
        info = h.info()
        g = L.ll_logdet_backward(h, dA, 1.0).cpu().numpy()
        res[kernel] = (est, g, info)
    assert res["tma"][2]["kernel_pass1"] == L.LL_KERNEL_TMA and res["tma"][2]["kernel_pass2"] == L.LL_KERNEL_TMA
    assert res["gather"][2]["kernel_pass2"] == L.LL_KERNEL_GATHER
    assert abs(res["tma"][0] - res["gather"][0]) <= 1e-12 * abs(res["gather"][0])
    # the TMA reverse step takes the gradient contraction into its tiles, where each entry's column
    # pairs are summed in another order than the separate contraction's: equal up to rounding
    gt, gg = res["tma"][1], res["gather"][1]
    assert np.max(np.abs(gt - gg)) <= 1e-12 * np.max(np.abs(gg))
    want = O.logdet_leja(A, lo, hi, 20, 30, 4, f32=(prec == "f32"))["estimate"]
    assert abs(res["tma"][0] - want) / abs(want) < TOL[prec]
    del torch


def test_autotuned_choice_is_cached_and_reported(L):
    A, lo, hi = _mat("lap3d_24")
    dA = L.DeviceCSR.from_host(A)
    h = L.Handle()
    opts = L.options(degree=15, probes=30, seed=2)
    e1 = L.ll_logdet_forward(h, dA, lo, hi, opts)
    i1 = h.info()
    e2 = L.ll_logdet_forward(h, dA, lo, hi, opts)
    i2 = h.info()
    assert i1["kernel_pass1"] in (L.LL_KERNEL_GATHER, L.LL_KERNEL_TMA)
    assert (i1["kernel_pass1"], i1["kernel_pass2"]) == (i2["kernel_pass1"], i2["kernel_pass2"])
    # the tuning launches happen on the first call only
    assert i2["kernel_launches"] < i1["kernel_launches"]
    assert e1 == e2


def test_tma_pipeline_wait_timeout_is_reported(L):
    """The stall hook leaves the first tile's pipeline phase incomplete (16 expected bytes that no
    copy delivers): the bounded waits run out, the kernel drains its issued copies and returns,
    the call fails with LL_ERR_TIMEOUT, and the handle and context stay usable."""
    A = laplacian_3d(32, 0.05)
    dA = L.DeviceCSR.from_host(A)
    h = L.Handle()
    h.debug_inject("stall")
    with pytest.raises(L.LejaError) as e:
        L.ll_logdet_forward(h, dA, 0.05, 12.05, L.options(degree=3, probes=30, seed=1, step_kernel="tma",
                                                             timeout_cycles=1_000_000, use_graph=False))
    assert e.value.name == "LL_ERR_TIMEOUT"
    h.debug_inject("none")
    est = L.ll_logdet_forward(h, dA, 0.05, 12.05, L.options(degree=3, probes=30, seed=1, step_kernel="tma"))
    ref = L.ll_logdet_forward(h, dA, 0.05, 12.05, L.options(degree=3, probes=30, seed=1, step_kernel="gather"))
    assert abs(est - ref) <= 1e-12 * abs(ref)


def test_graph_replay_matches_eager(L):
    """An identical second call replays the captured CUDA graph: same estimate, same phase
    events, same launch count; any change of inputs (seed, values in place) is seen. The step
    kernel is fixed so that two handles run the same kernels (the autotuner times candidates and
    may choose differently per handle)."""
    A, lo, hi = _mat("lap3d_24")
    dA = L.DeviceCSR.from_host(A)
    h = L.Handle()
    opts = L.options(degree=15, probes=30, seed=2, use_graph=True, step_kernel="tma")
    e1 = L.ll_logdet_forward(h, dA, lo, hi, opts)   # eager, then captured
    i1 = h.info()
    e2 = L.ll_logdet_forward(h, dA, lo, hi, opts)   # replay
    i2 = h.info()
    e3 = L.ll_logdet_forward(h, dA, lo, hi, opts)   # replay
    h2 = L.Handle()
    eg = L.ll_logdet_forward(h2, dA, lo, hi, L.options(degree=15, probes=30, seed=2, use_graph=False, step_kernel="tma"))
    assert e1 == e2 == e3 == eg
    assert i2["ms_pass1"] > 0 and i2["ms_pass2"] > 0 and i2["ms_total"] >= i2["ms_pass2"]
    assert i2["kernel_launches"] == i1["kernel_launches"]
    assert (i2["kernel_pass1"], i2["kernel_pass2"]) == (i1["kernel_pass1"], i1["kernel_pass2"])
    o3 = L.options(degree=15, probes=30, seed=3, use_graph=True, step_kernel="tma")
    e4 = L.ll_logdet_forward(h, dA, lo, hi, o3)
    e4g = L.ll_logdet_forward(h2, dA, lo, hi, L.options(degree=15, probes=30, seed=3, use_graph=False, step_kernel="tma"))
    assert e4 == e4g and e4 != e1
    # values changed in place (same pointers): the replay reads the new values
    dA.values.mul_(2.0)
    L.ll_logdet_forward(h, dA, 2 * lo, 2 * hi, o3)
    e5 = L.ll_logdet_forward(h, dA, 2 * lo, 2 * hi, o3)
    e5g = L.ll_logdet_forward(h2, dA, 2 * lo, 2 * hi, L.options(degree=15, probes=30, seed=3, use_graph=False, step_kernel="tma"))
    assert e5 == e5g


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("b", [1, 2, 7, 33, 66])
@pytest.mark.parametrize("threads", [512, 256])
def test_tma_two_pairs_per_thread_matches_gather_bitwise(L, name, b, threads):
    """FP32-mixed, two column pairs per consumer thread (one 16-byte access per operand row and
    twice the rows per tile): the same per-column arithmetic in the same entry order, so p(A)V
    equals the register kernel's bit for bit, including the pad columns of widths that are not
    multiples of four and the ragged last tile."""
    A, lo, hi = _mat(name)
    V = R.rademacher(7, R.STREAM_S, A.n, b)
    g, _ = _apply(L, A, lo, hi, 12, V, "f32", "gather")
    t, it = _apply(L, A, lo, hi, 12, V, "f32", "tma", threads=threads, rpt=2)
    assert it["kernel_pass1"] == L.LL_KERNEL_TMA and it["pairs_pass1"] == 2
    assert np.array_equal(g, t)


def test_tma_two_pairs_per_thread_forward_and_backward(L):
    """The trace pass (DOT), the adjoint's recompute (PLAIN) and reverse (ADJ) steps with two
    column pairs per thread: the estimate equals the one-pair kernel's to rounding (the traces
    are summed over another row grouping), and so do the value gradients (the one-pair reverse
    step takes the gradient contraction into its tiles and sums each entry's column pairs in
    another order than the separate contraction that follows the two-pair step)."""
    need_gpu()
    A, lo, hi = _mat("matern_60")
    dA = L.DeviceCSR.from_host(A, "f32")
    res = {}
    for rpt in (0, 2):
        h = L.Handle()
        h.set_step_config("tma", 0, rpt)
        est = L.ll_logdet_forward(h, dA, lo, hi, L.options(degree=20, probes=30, seed=4, precision="f32",
                                                              keep_for_backward=True, step_kernel="tma",
                                                              rows_per_thread=rpt))
        info = h.info()
        assert info["pairs_pass1"] == info["pairs_pass2"] == (2 if rpt == 2 else 1)
        res[rpt] = (est, L.ll_logdet_backward(h, dA, 1.0).cpu().numpy())
    assert abs(res[2][0] - res[0][0]) <= 1e-12 * abs(res[0][0])
    assert np.max(np.abs(res[2][1] - res[0][1])) <= 1e-12 * np.max(np.abs(res[0][1]))
    want = O.logdet_leja(A, lo, hi, 20, 30, 4, f32=True)["estimate"]
    assert abs(res[2][0] - want) / abs(want) < TOL["f32"]
