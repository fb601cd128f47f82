"""torch.autograd face of the gated operator A_i = A D_{u_i} (Sec. II-A).

Forward: y = A D_{u_i} x through mc_forward (after mc_set_field when a field
is given).  Backward: one mc_vjp call gives both x's gradient, the matched
adjoint A_i^* g (D_i^T A^T g, exact transpose of the forward kernels), and the
field's gradient, g backprojected and multiplied by the spatial derivative of
the bilinear sample at p + u_i(p).  Both run in libmc's kernels; there is no
PyTorch fallback.

The context holds one field per gate.  If the gate's field was replaced
between forward and backward, backward puts the saved field back for its
mc_vjp call and then restores the field that was current before, so a graph
always differentiates the operator its forward applied and later users of the
context see the field most recently set.  Each replacement rebuilds the gate's
D_i^T and, as every mc_set_field does, drops the context's norms and step sizes.
"""
from __future__ import annotations

import torch


class GateProjection(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ctx, gate: int, x, field):
        if not (x.is_cuda and x.dtype == torch.float32):
            raise TypeError("x must be a float32 CUDA tensor")
        x = x.contiguous()
        if field is not None:
            if not (field.is_cuda and field.dtype == torch.float32):
                raise TypeError("field must be a float32 CUDA tensor")
            field = field.contiguous()
            ctx.set_field(gate, field.detach())
        y = ctx.forward(gate, x.detach())
        fctx.mc = ctx
        fctx.gate = gate
        fctx.version = ctx.field_version(gate)
        fctx.has_field = field is not None
        fctx.save_for_backward(x, field if field is not None else x.new_empty(0))
        return y

    @staticmethod
    def backward(fctx, gy):
        x, field = fctx.saved_tensors
        ctx, gate = fctx.mc, fctx.gate
        need_x = fctx.needs_input_grad[2]
        need_f = fctx.has_field and fctx.needs_input_grad[3]
        if not (need_x or need_f):
            return None, None, None, None
        if fctx.has_field and ctx.field_version(gate) != fctx.version:
            now = ctx.current_field(gate)
            ctx.set_field(gate, field.detach())
            try:
                gx, gf = ctx.vjp(gate, x.detach(), gy.contiguous(), grad_x=need_x, grad_field=need_f)
            finally:
                ctx.set_field(gate, now)
            return None, None, gx, gf
        gx, gf = ctx.vjp(gate, x.detach(), gy.contiguous(), grad_x=need_x, grad_field=need_f)
        return None, None, gx, gf
