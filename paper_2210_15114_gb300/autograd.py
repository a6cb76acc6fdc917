"""torch.autograd access to the distance-matrix product.

``DistanceProduct.apply(X, Z, metric, ctx)`` returns A(X) Z through the C ABI
(dm_prepare + dm_matmat).  Its backward pass is also two C-ABI calls:
  * dL/dX = dm_grad(plan, W = dL/dout, Z), the gradient of
    sum_q w_q^T A(X) z_q (sgn(0) = 0 at tied coordinates for l1);
  * dL/dZ = A^T dL/dout = A dL/dout (A is symmetric), one more dm_matmat.
Nothing here computes: the module only routes tensors to the library.
Both passes issue their work on torch's current stream (the context is
switched to it when it differs) and end with dm_sync, so a device-side error
(a bounded wait that ran out, non-finite coordinates) raises here instead of
leaving a wrong result behind.
"""
from __future__ import annotations

import torch

from . import binding


def _follow_current_stream(dmctx, device):
    if device.type != "cuda":
        return                        # the library rejects the tensors itself
    s = torch.cuda.current_stream(device).cuda_stream
    if getattr(dmctx, "stream", None) != s:
        binding.dm_set_stream(dmctx, s)


class DistanceProduct(torch.autograd.Function):
    @staticmethod
    def forward(fctx, X, Z, metric, dmctx):
        _follow_current_stream(dmctx, X.device)
        plan = binding.dm_prepare(dmctx, metric, X)
        out = binding.dm_matmat(plan, Z)
        binding.dm_sync(dmctx)
        fctx.plan = plan
        fctx.dmctx = dmctx
        fctx.save_for_backward(X, Z)
        return out

    @staticmethod
    def backward(fctx, grad_out):
        X, Z = fctx.saved_tensors
        plan = fctx.plan
        _follow_current_stream(fctx.dmctx, X.device)
        g = grad_out.contiguous()
        gX = gZ = None
        if fctx.needs_input_grad[0]:
            gX = binding.dm_grad(plan, g, Z.contiguous())
        if fctx.needs_input_grad[1]:
            gZ = binding.dm_matmat(plan, g)
        binding.dm_sync(fctx.dmctx)
        return gX, gZ, None, None


_default_ctx = {}


def distance_product(X, Z, metric: str = "l1", ctx=None):
    """A(X) Z with autograd support (X: n x d, Z: n or n x k, same device)."""
    if ctx is None:
        dev = X.device.index or 0
        if dev not in _default_ctx:
            _default_ctx[dev] = binding.dm_create(dev)
        ctx = _default_ctx[dev]
    return DistanceProduct.apply(X, Z, metric, ctx)
