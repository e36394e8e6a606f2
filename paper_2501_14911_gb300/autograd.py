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


class EllipticOp(torch.autograd.Function):
    """u = A_s m per time block (the elliptic prior operator of Eq. (5.1)); A_s is
    symmetric, so the backward pass applies A_s again."""

    @staticmethod
    def forward(ctx, m, handle, gx, gy, alpha1, alpha2):
        m = m.contiguous()
        out = torch.empty_like(m)
        handle.apply_elliptic(gx, gy, alpha1, alpha2, m, out)
        ctx.args = (handle, gx, gy, alpha1, alpha2)
        return out

    @staticmethod
    def backward(ctx, g):
        handle, gx, gy, alpha1, alpha2 = ctx.args
        g = g.contiguous()
        out = torch.empty_like(g)
        handle.apply_elliptic(gx, gy, alpha1, alpha2, g, out)
        return out, None, None, None, None, None


def map_loss(handle, m, d, sigma2, gx, gy, alpha1=1.0, alpha2=1.0):
    """0.5 ||F m - d||^2 / sigma2 + 0.5 sum_t ||A_s m_t||^2 with gradients through the
    library's F^T and elliptic kernels (the negative log-posterior of Sec. 2 with the
    elliptic prior of Eq. (5.1))."""
    r = FOp.apply(m, handle) - d
    u = EllipticOp.apply(m, handle, gx, gy, alpha1, alpha2)
    return 0.5 * (r * r).sum() / sigma2 + 0.5 * (u * u).sum()
