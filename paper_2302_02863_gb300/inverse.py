"""Inverse-problem outer loop on top of the differentiable solve: recover the
nodal fractional order s (log kappa known) from an observed solution u_obs
by minimising the misfit

    J(s) = || U(s) - u_obs ||^2_{M_L},    A(s, log kappa) U(s) = F,

with ||e||^2_{M_L} = sum_i m_i e_i^2 the lumped P1 mass norm (m = M_0 1), by
projected gradient descent with Armijo backtracking; s is kept in
[s_min, s_max] inside the quadrature bound s_bar of Sec. 4.  The paper stops at
the forward problem and names the inverse problem as the next step (Sec. 8);
every solve and gradient runs in libvfd.so through autograd.solve (adjoint
solve + vfd_grad, exact for the H^2 operator the solve uses).
"""
from __future__ import annotations

import torch

from . import autograd, vfd


def lumped_mass(mesh, n_vert, device="cuda"):
    """m = M_0 1 on the DoFs: the row sums of the P1 mass matrix."""
    F = torch.zeros(mesh.n_dof, dtype=torch.float64, device=device)
    vfd.vfd_load(mesh, torch.ones(n_vert, dtype=torch.float64, device=device), F)
    return F


def misfit(s, logk, F, u_obs, m_lumped, mesh, s_bar):
    U = autograd.solve(s, logk, F, mesh, s_bar)
    e = U - u_obs
    return (m_lumped * e * e).sum()


def fit_order(mesh, n_vert, F, u_obs, s0, logk, s_bar=0.9, steps=10, step0=1.0, s_min=0.05, s_max=None,
              armijo=1e-4, shrink=0.5, max_backtrack=12):
    """Projected gradient descent on the nodal s (float64 CUDA tensor of
    n_vert values); returns (s, history of J at the accepted iterates).  The
    first trial step is scaled so that it moves s by step0 * 0.1 at most."""
    s_max = s_bar if s_max is None else s_max
    m_l = lumped_mass(mesh, n_vert, F.device)
    s = s0.detach().clone().clamp(s_min, s_max)
    hist = []
    for _ in range(steps):
        s_var = s.clone().requires_grad_(True)
        J = misfit(s_var, logk, F, u_obs, m_l, mesh, s_bar)
        (g,) = torch.autograd.grad(J, s_var)
        J0 = J.item()
        hist.append(J0)
        gmax = g.abs().max().item()
        if gmax == 0.0:
            break
        t = step0 * 0.1 / gmax
        accepted = False
        for _ in range(max_backtrack):
            s_new = (s - t * g).clamp(s_min, s_max)
            with torch.no_grad():
                J1 = misfit(s_new, logk, F, u_obs, m_l, mesh, s_bar).item()
            if J1 <= J0 - armijo * (g * (s - s_new)).sum().item():
                accepted = True
                break
            t *= shrink
        if not accepted:
            break
        s = s_new.detach()
    return s, hist
