"""``torch.autograd.Function`` over the SLR row bounds of a batch of boxes.

Forward returns the float32 SLR lower and upper bounds of every property row
(Sec. 2.2, Eq. 1; Sec. 3) for each box; backward calls the library's adjoint
kernel (``slr_margin_backward``) with the incoming gradients and returns the
gradients with respect to the box endpoints, the lower ReLU slopes (when they
are given) and, when the weight tensors are passed, the weights and biases.
PyTorch only carries the tensors; both directions run in the library's CUDA
kernels.
"""
from __future__ import annotations

import torch

from . import slr_margin_backward


class SLRRowBounds(torch.autograd.Function):
    """lo, hi = SLRRowBounds.apply(counter, box_lo, box_hi, alpha, *W, *b).

    counter: a ``Counter`` with network and property set.  box_lo, box_hi:
    (n, d) CUDA float32 tensors.  alpha: (n, H) slopes or None (then the slopes
    are u/(u-l) and gradients flow through that formula).  W, b: optional
    weight and bias tensors of the network (K of each, in the network's own
    shapes); when given they are loaded into the counter and receive gradients.
    """

    @staticmethod
    def forward(fctx, counter, box_lo, box_hi, alpha, *params):
        K = len(params) // 2
        if K:
            counter.load_network([w.detach().float().cpu().numpy() for w in params[:K]],
                                 [x.detach().float().cpu().numpy() for x in params[K:]])
        n, R = int(box_lo.shape[0]), counter.R
        z = torch.zeros((n, R), dtype=torch.float32, device=box_lo.device)
        out = slr_margin_backward(counter.ctx, box_lo, box_hi, R, z, z, alpha, None, want_rows=True,
                                  want_alpha=False, want_box=False)
        fctx.counter = counter
        fctx.K = K
        fctx.has_alpha = alpha is not None
        fctx.save_for_backward(box_lo, box_hi, alpha if alpha is not None else z)
        return out["row_lo"], out["row_hi"]

    @staticmethod
    def backward(fctx, g_lo, g_hi):
        box_lo, box_hi, alpha = fctx.saved_tensors
        counter = fctx.counter
        R = counter.R
        g_lo = torch.zeros_like(box_lo[:, :1].expand(-1, R)) if g_lo is None else g_lo
        g_hi = torch.zeros_like(box_lo[:, :1].expand(-1, R)) if g_hi is None else g_hi
        out = slr_margin_backward(counter.ctx, box_lo, box_hi, R, g_lo.float().contiguous(),
                                  g_hi.float().contiguous(), alpha if fctx.has_alpha else None,
                                  counter.widths if fctx.K else None, want_rows=False,
                                  want_alpha=fctx.has_alpha, want_box=True)
        grads = [None, out["d_lo"], out["d_hi"], out["d_alpha"] if fctx.has_alpha else None]
        if fctx.K:
            grads += list(out["d_W"]) + list(out["d_b"])
        return tuple(grads)
