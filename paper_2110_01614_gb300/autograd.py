"""torch.autograd.Function over the nsdf query and its hand-written backward.

``sdf_query(pts, blob, net)`` returns (f, grad f) for points [n, 4] and a
weight blob (float32 vector in the packed layout); gradients of any loss of f
and grad f flow to the points and to the blob through nsdf_backward (FP32
kernel, activations recomputed per tile).  ``net`` is a NeuralSDF context of
FP32 precision whose weights are (re)loaded from ``blob`` on every call, so
the blob can be a trainable parameter.
"""

import torch

from . import NSDF_RAW_GRADIENT, nsdf_backward, nsdf_query


class SDFQuery(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pts, blob, net):
        # an output the loss does not use gets no gradient (None, not zeros),
        # so a loss of f alone takes the first-order path of nsdf_backward
        ctx.set_materialize_grads(False)
        net.load(blob.detach())
        out = torch.empty_like(pts)
        nsdf_query(net.ctx, pts, out, NSDF_RAW_GRADIENT)
        ctx.save_for_backward(pts)
        ctx.net = net
        return out[:, 3].contiguous(), out[:, :3].contiguous()

    @staticmethod
    def backward(ctx, g_f, g_grad):
        (pts,) = ctx.saved_tensors
        net = ctx.net
        n = pts.shape[0]
        a = g_f.contiguous() if g_f is not None else torch.zeros(n, device=pts.device)
        v = None
        if g_grad is not None:
            v = torch.zeros(n, 4, device=pts.device, dtype=torch.float32)
            v[:, :3] = g_grad
        need_p, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        g_w = None
        if need_w:
            from . import nsdf_num_params
            g_w = torch.empty(nsdf_num_params(net.arch), device=pts.device, dtype=torch.float32)
        g_p = torch.empty_like(pts) if need_p else None
        if g_w is None and g_p is None:
            return None, None, None
        if g_p is None and v is None:
            g_p = torch.empty_like(pts)            # the first-order path writes points
        nsdf_backward(net.ctx, pts, a, v, g_w, g_p)
        return (g_p if need_p else None), g_w, None


def sdf_query(pts, blob, net):
    return SDFQuery.apply(pts, blob, net)
