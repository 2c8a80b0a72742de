"""torch.autograd.Function over the C ABI: U = A(s, log kappa)^{-1} F with P1
(nodal) fields s and log kappa.

Argument marshalling only: the forward pass calls vfd_assemble and vfd_solve,
the backward pass the adjoint solve (A is symmetric: A Lam = dL/dU) and
vfd_grad, which returns -Lam^T (dA/dtheta) U for theta = nodal s and nodal
log kappa; dL/dF = Lam.  Every step runs in libvfd.so on the device.
"""
from __future__ import annotations

import torch

from . import vfd


class _Nodal:
    """A P1 field given by its vertex values (device tensor)."""

    def __init__(self, values):
        self.nodal = values


class VfdSolve(torch.autograd.Function):
    """U = VfdSolve.apply(s, logk, F, mesh, s_bar, rtol, max_it).

    s, logk: float64 CUDA tensors of n_vert vertex values; F: float64 CUDA
    tensor (n_dof,) or (nrhs, n_dof).  Any admissibility (the gradient is
    that of the H^2 operator the solve uses, P1 fields at the Chebyshev
    nodes by the nearest-point rule); tail_mode 0."""

    @staticmethod
    def forward(ctx, s, logk, F, mesh, s_bar=0.9, rtol=1e-12, max_it=100000):
        s_c = s.detach().contiguous()
        k_c = logk.detach().contiguous()
        op = vfd.vfd_assemble(mesh, _Nodal(s_c), _Nodal(k_c), s_bar)
        F_c = F.detach().contiguous()
        U = torch.zeros_like(F_c)
        vfd.vfd_solve(op, F_c, U, rtol=rtol, max_it=max_it, raise_on_noconv=True)
        ctx.op = op
        ctx.rtol, ctx.max_it = rtol, max_it
        ctx.save_for_backward(U)
        return U

    @staticmethod
    def backward(ctx, gU):
        (U,) = ctx.saved_tensors
        op = ctx.op
        Lam = torch.zeros_like(U)
        vfd.vfd_solve(op, gU.contiguous(), Lam, rtol=ctx.rtol, max_it=ctx.max_it, raise_on_noconv=True)
        n_vert = op.mesh.info["n_vert"]
        g_s = torch.empty(n_vert, dtype=torch.float64, device=U.device)
        g_k = torch.empty_like(g_s)
        vfd.vfd_grad(op, U, Lam, g_s, g_k)
        return g_s, g_k, Lam, None, None, None, None


def solve(s, logk, F, mesh, s_bar=0.9, rtol=1e-12, max_it=100000):
    """Differentiable solve; see VfdSolve."""
    return VfdSolve.apply(s, logk, F, mesh, s_bar, rtol, max_it)
