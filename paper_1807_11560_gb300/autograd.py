"""torch.autograd interface to the shoot-and-transport map v0 -> m(1).

``shoot_transport(ctx, v0)`` returns m(1) (Eqs. 51-52 on the GPU); its
backward is one of the library's hand-written adjoint sweeps, so any loss
built on m(1) in PyTorch differentiates through the band-limited EPDiff
shoot without storing a torch graph of the sweep:

* ``adjoint="jacobi"`` (default): the paper's reduced adjoint Jacobi sweep
  (``lddmm_transport_vjp``, Eqs. 53-55 with the loss gradient in place of the
  data term), the gradient the method's Gauss-Newton-Krylov solver uses;
* ``adjoint="exact"``: the exact discrete adjoint of the discretised map
  (``lddmm_transport_vjp_exact``, the route of Eqs. 12-14 in discrete form),
  the true derivative of the computed m(1) (what finite differences see).

The backward recomputes the forward trajectory from v0 (v0 is the only
checkpoint kept by autograd).
"""

import torch

__all__ = ["ShootTransport", "shoot_transport"]


class ShootTransport(torch.autograd.Function):
    @staticmethod
    def forward(fctx, v0, ctx, adjoint="jacobi"):
        if adjoint not in ("jacobi", "exact"):
            raise ValueError("adjoint is 'jacobi' or 'exact'")
        m1 = torch.empty(ctx.grid, dtype=torch.float64 if ctx.precision == "fp64" else torch.float32,
                         device=v0.device)
        ctx.transport(v0.detach().contiguous(), m1)
        fctx.lddmm = ctx
        fctx.exact = adjoint == "exact"
        fctx.save_for_backward(v0)
        return m1

    @staticmethod
    def backward(fctx, grad_m1):
        (v0,) = fctx.saved_tensors
        g = torch.empty_like(v0)
        fctx.lddmm.transport_vjp(v0.detach().contiguous(), grad_m1.contiguous(), g, exact=fctx.exact)
        return g, None, None


def shoot_transport(ctx, v0, adjoint="jacobi"):
    """m(1) for band-limited v0 [d][K..] (complex), differentiable in v0 through
    the adjoint sweep named by ``adjoint`` ("jacobi" or "exact")."""
    return ShootTransport.apply(v0, ctx, adjoint)
