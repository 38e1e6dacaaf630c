"""The allocation-free power iteration (collected last on purpose).

ll_power_lmax_noalloc exists for callers that cannot allocate device memory: code whose device
memory belongs to another allocator, or code that cannot afford the implicit synchronisation of
cudaMalloc/cudaFree. It runs the kernels of the allocating entry point with the same grid and
reduction order, so it must return exactly what that entry point returns, call after call,
although every call reuses the same library-owned scratch array; and it must not take device
memory.
"""
from __future__ import annotations

import pytest

from synth import laplacian_2d, random_spd
from tests.gpu_util import lib

pytestmark = pytest.mark.gpu


def test_noalloc_power_iteration_matches_allocating_entry_point():
    L = lib()
    h = L.Handle()
    cases = [(random_spd(5000, seed=7), 20, 3), (laplacian_2d(300, 0.1), 20, 1), (random_spd(1234, seed=2), 7, 5)]
    for A, iters, seed in cases:
        dA = L.DeviceCSR.from_host(A)
        want = L.ll_power_lmax(h, dA, iters=iters, seed=seed)
        for _ in range(2):                       # two calls in a row reuse the same scratch
            got = L.ll_power_lmax_noalloc(dA, iters=iters, seed=seed)
            assert got == want                   # same kernels, grid and summation order


def test_noalloc_power_iteration_takes_no_device_memory():
    import torch
    L = lib()
    A = laplacian_2d(400, 0.1)
    dA = L.DeviceCSR.from_host(A)
    L.ll_power_lmax_noalloc(dA, iters=5, seed=0)    # first call: the scratch address is looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    vals = [L.ll_power_lmax_noalloc(dA, iters=20, seed=s) for s in range(10)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # any workspace allocation takes at least one 2 MiB page of device memory
    assert free0 - free1 < (1 << 20), (free0, free1)
    assert all(v > 0 for v in vals)


def test_noalloc_power_iteration_rejects_too_many_rows():
    L = lib()
    A = laplacian_2d(513, 0.1)                   # 263,169 rows > 262,144
    dA = L.DeviceCSR.from_host(A)
    with pytest.raises(L.LejaError) as ei:
        L.ll_power_lmax_noalloc(dA, iters=3, seed=0)
    assert ei.value.name == "LL_ERR_UNSUPPORTED"
