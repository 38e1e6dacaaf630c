"""Seeded synthetic inputs shared by the oracle-side tests, the CUDA-side tests and the bench.

This package only builds input data (sparse SPD matrices in CSR form and the parameters of
batched workloads). It holds none of the log-determinant method's arithmetic: no bounds, no
Léja points, no divided differences, no probes, no recurrence.
"""
from .matrices import (  # noqa: F401
    CSR,
    laplacian_2d,
    laplacian_3d,
    matern_2d,
    matern_2d_derivatives,
    gmrf_batch_params,
    powerlaw_laplacian,
    pentadiagonal,
    gmrf_theta,
    diagonal,
    random_spd,
    csr_from_dense,
)
