"""The inverse-problem outer loop (paper_2302_02863_gb300.inverse.fit_order)
on the GPU against the same projected-gradient loop run with the oracle's
dense matrices: dense solves for U and the adjoint, oracle.grad for
-Lam^T (dA/ds) U.  Both follow the same step rule, so the misfit history
and the final nodal s must agree to the solve tolerance; the misfit must
decrease at every accepted step and by two orders of magnitude over eight.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import autograd, inverse, vfd  # noqa: E402

SBAR = 0.9
STEPS = 8


def _fields(m):
    x = m.coords
    s_true = 0.45 + 0.12 * np.sin(2.0 * x[:, 0]) + 0.08 * np.cos(1.7 * x[:, 1])
    lk = 0.2 * np.cos(1.5 * x[:, 1])
    return s_true, lk


def _oracle_loop(m, s_true, lk, s0):
    F = oracle.load(m, np.ones(m.n_vert))
    m_l = F.copy()

    def solve(s):
        ref = oracle.assemble(m, synth.nodal_field(s), synth.nodal_field(lk), s_bar=SBAR, n_sing=3)
        return ref, oracle.cholesky_solve(ref.A, F)

    u_obs = solve(s_true)[1]

    def J(s):
        ref, U = solve(s)
        e = U - u_obs
        return (m_l * e * e).sum(), ref, U, e

    s, hist = s0.copy(), []
    for _ in range(STEPS):
        j, ref, U, e = J(s)
        hist.append(j)
        Lam = oracle.cholesky_solve(ref.A, 2.0 * m_l * e)
        g = oracle.grad(m, s, lk, U[None], Lam[None], s_bar=SBAR, n_sing=3)[0]
        t = 0.1 / np.abs(g).max()
        for _ in range(12):
            s_new = np.clip(s - t * g, 0.05, SBAR)
            if J(s_new)[0] <= j - 1e-4 * (g * (s - s_new)).sum():
                break
            t *= 0.5
        s = s_new
    return np.array(hist), s


def test_fit_order_follows_oracle_loop():
    m = synth.disk_mesh(5, R=1.1, jitter=0.2, seed=8)
    s_true, lk = _fields(m)
    s0 = np.full(m.n_vert, 0.5)
    hist_o, s_o = _oracle_loop(m, s_true, lk, s0)

    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=16, lam=0.0, rho_lambda=0.0)
    dev = "cuda"
    F = torch.zeros(mesh.n_dof, dtype=torch.float64, device=dev)
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device=dev), F)
    lk_t = torch.tensor(lk, device=dev)
    with torch.no_grad():
        u_obs = autograd.solve(torch.tensor(s_true, device=dev), lk_t, F, mesh, SBAR)
    s, hist = inverse.fit_order(mesh, m.n_vert, F, u_obs, torch.tensor(s0, device=dev), lk_t, s_bar=SBAR,
                                steps=STEPS)
    hist = np.array(hist)
    assert len(hist) == STEPS
    assert np.all(np.diff(hist) < 0)
    assert hist[-1] < 0.05 * hist[0]
    assert np.abs(hist - hist_o).max() / hist_o[0] < 1e-7, (hist, hist_o)
    assert np.abs(s.cpu().numpy() - s_o).max() < 1e-6
