"""F as a torch.autograd.Function: forward is libbti's F kernel path, backward
its exact transpose F^T (Sec. 4: the adjoint uses the conjugate-transposed
spectral blocks).  The gradient of 0.5 ||F m - d||^2_{Gamma_n^{-1}} with
respect to m is F^T Gamma_n^{-1} (F m - d), so autograd reaches it through
one apply_F and one apply_FT call."""

import torch


class FOp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, handle):
        m = m.contiguous()
        d = torch.empty(m.shape[:-2] + (handle.Nt, handle.Nd), dtype=m.dtype, device=m.device)
        handle.apply_F(m, d)
        ctx.handle = handle
        return d

    @staticmethod
    def backward(ctx, grad_d):
        h = ctx.handle
        g = grad_d.contiguous()
        gm = torch.empty(g.shape[:-2] + (h.Nt, h.Nm), dtype=g.dtype, device=g.device)
        h.apply_FT(g, gm)
        return gm, None


def apply_F_autograd(handle, m):
    """d = F m with gradients flowing through F^T."""
    return FOp.apply(m, handle)
