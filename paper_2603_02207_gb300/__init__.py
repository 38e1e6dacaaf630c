"""GB300-native Léja-point log-determinant estimator (arXiv 2603.02207).

The compute path is the native library libleja.so (CUDA for sm_103a behind the C ABI in
include/leja.h); this package is its thin Python binding. Importing the package does not load
the library; the first call does, and raises ImportError if it has not been built.
"""
from .api import (DeviceCSR, Handle, LejaError, ll_apply_poly, ll_apply_poly_tol, ll_divided_differences,  # noqa: F401
                  ll_divided_differences_q,
                  ll_gershgorin, ll_leja_points, ll_logdet_backward, ll_logdet_forward,
                  ll_kept_basis, ll_logdet_batched, ll_logdet_sweep, ll_logdet_forward_host, ll_param_grad, ll_power_lmax, ll_power_lmax_noalloc, ll_probes, logdet_leja,
                  ll_stop_degrees, options, ll_gram, df64_block)
from .api import LL_EST_HUTCHINSON, LL_EST_HUTCHPP, LL_KERNEL_AUTO, LL_KERNEL_BAND, LL_KERNEL_GATHER, LL_KERNEL_TMA, STEP_KERNELS  # noqa: F401
from .autograd import LejaLogdet, logdet  # noqa: F401
