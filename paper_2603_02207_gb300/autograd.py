"""torch.autograd.Function over the C ABI: the Léja/Hutch++ log-determinant estimate as a
differentiable function of the stored CSR values.

The backward is the library's adjoint: by default (ll_logdet_backward) the derivative of the
estimate with the Hutch++ basis [Q | G'], the spectral bounds, sigma and the Newton coefficients
held fixed; with through_qr=True (ll_logdet_backward_qr) the exact derivative of the estimate,
the sketch's QR included (the bounds, sigma and the coefficients still fixed).
Gradients with respect to model parameters follow from torch's chain rule when the values are a
torch expression of those parameters, or from ll_param_grad given d values / d theta.
"""
from __future__ import annotations

import torch

from . import api


class LejaLogdet(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, rowptr, colind, n, lmin, lmax, degree, probes, seed, precision, probe_kind, handle,
                through_qr=False):
        A = api.DeviceCSR(n=int(n), rowptr=rowptr, colind=colind, values=values.detach().contiguous())
        opts = api.options(degree=degree, probes=probes, seed=seed, precision=precision, probe_kind=probe_kind,
                           keep_for_backward=True)
        est = api.ll_logdet_forward(handle, A, lmin, lmax, opts)
        ctx.forward_id = handle.info()["forward_id"]
        ctx.handle = handle
        ctx.A = A
        ctx.through_qr = bool(through_qr)
        return torch.tensor(est, dtype=torch.float64, device=values.device)

    @staticmethod
    def backward(ctx, grad_out):
        # the handle keeps the state of its last forward only: refuse to differentiate an older one
        if ctx.handle.info()["forward_id"] != ctx.forward_id:
            raise api.LejaError(11, "another forward ran on this handle since this estimate's "
                                    "(one handle per differentiable estimate)")
        g = api.ll_logdet_backward(ctx.handle, ctx.A, float(grad_out), through_qr=ctx.through_qr)
        return g.to(ctx.A.values.dtype), None, None, None, None, None, None, None, None, None, None, None, None


def logdet(values, rowptr, colind, n: int, bounds: tuple[float, float], degree: int, probes: int, seed: int = 0,
           precision: str = "df64", probe_kind: str = "rademacher", handle: api.Handle | None = None,
           through_qr: bool = False):
    """Differentiable logdet_leja(csr, bounds, degree, probes, seed) of the CSR matrix
    (rowptr, colind, values) on the current CUDA device; values may require grad. through_qr:
    differentiate through the sketch's QR too (the exact derivative of the estimate)."""
    h = handle or api.Handle()
    return LejaLogdet.apply(values, rowptr, colind, n, bounds[0], bounds[1], degree, probes, seed, precision,
                            probe_kind, h, through_qr)
