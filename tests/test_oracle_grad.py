"""Pins of the oracle's adjoint gradient (derivative of the discrete matrix
with respect to nodal s and log kappa; the paper has no gradients, the
method is the adjoint rule g = -Lam^T (dA/dtheta) U with A Lam = dJ/dU).

* central finite differences of J(theta) = Lam0^T U(theta), U = A^{-1} F,
  along random and single-vertex directions, with A re-assembled by the
  oracle's assembly routine and solved by its Cholesky: a route that shares
  only the quadrature with the gradient loops, so a dropped term, a wrong
  sign or a wrong basis weight in the gradient shows up;
* the uniform shift of log kappa scales every term of A by e^c, so the
  log-kappa gradient sums to -Lam^T A U exactly;
* linearity in the right-hand sides.
"""
import numpy as np
import pytest

import oracle
import synth

SBAR, NS = 0.9, 3


def _fields(m, seed):
    rng = np.random.default_rng(seed)
    x = m.coords
    s = 0.45 + 0.15 * np.sin(2.0 * x[:, 0]) + 0.05 * rng.standard_normal(m.n_vert)
    lk = 0.3 * np.cos(1.5 * x[:, -1]) + 0.1 * rng.standard_normal(m.n_vert)
    return np.clip(s, 0.15, 0.8), lk


def _solve(m, s, lk, F):
    A = oracle.assemble(m, synth.nodal_field(s), synth.nodal_field(lk), s_bar=SBAR, n_sing=NS)
    return A, oracle.cholesky_solve(A.A, F)


def _check_fd(m, seed, n_dirs=3, h=1e-6, tol=1e-6):
    s, lk = _fields(m, seed)
    F = oracle.load(m, np.ones(m.n_vert))
    rng = np.random.default_rng(seed + 1)
    A, U = _solve(m, s, lk, F)
    lam0 = rng.standard_normal(A.N)
    Lam = oracle.cholesky_solve(A.A, lam0)
    gs, gk = oracle.grad(m, s, lk, U, Lam, s_bar=SBAR, n_sing=NS)
    dirs = [rng.standard_normal(m.n_vert) for _ in range(n_dirs)]
    # single vertices: an interior DoF and a vertex of the exterior layer
    e = np.zeros(m.n_vert)
    e[np.nonzero(A.dof >= 0)[0][len(np.nonzero(A.dof >= 0)[0]) // 2]] = 1.0
    dirs.append(e)
    e = np.zeros(m.n_vert)
    e[np.nonzero(A.dof < 0)[0][0]] = 1.0
    dirs.append(e)
    for which, g in (("s", gs), ("logk", gk)):
        for v in dirs:
            if which == "s":
                Jp = lam0 @ _solve(m, s + h * v, lk, F)[1]
                Jm = lam0 @ _solve(m, s - h * v, lk, F)[1]
            else:
                Jp = lam0 @ _solve(m, s, lk + h * v, F)[1]
                Jm = lam0 @ _solve(m, s, lk - h * v, F)[1]
            fd = (Jp - Jm) / (2 * h)
            ad = g @ v
            assert abs(ad - fd) <= tol * max(abs(fd), 1e-3 * np.abs(g).sum() * np.abs(v).max()), (which, ad, fd)


def test_grad_matches_finite_differences_2d():
    _check_fd(synth.disk_mesh(3, R=1.1, jitter=0.2, seed=5), seed=11)


def test_grad_matches_finite_differences_1d():
    _check_fd(synth.interval_mesh(12, R=1.2), seed=12)


def test_logk_shift_invariant():
    # gamma scales by e^c under logk -> logk + c, so A -> e^c A and
    # sum_k dA/dlogk_k = A: the log-kappa gradient sums to -Lam^T A U
    m = synth.disk_mesh(4, R=1.1, jitter=0.2, seed=6)
    s, lk = _fields(m, 21)
    F = oracle.load(m, np.ones(m.n_vert))
    A, U = _solve(m, s, lk, F)
    Lam = np.random.default_rng(3).standard_normal(A.N)
    gs, gk = oracle.grad(m, s, lk, U, Lam, s_bar=SBAR, n_sing=NS)
    ref = -(Lam @ (A.A @ U))
    assert abs(gk.sum() - ref) <= 1e-11 * abs(ref)


def test_grad_linear_in_columns():
    m = synth.disk_mesh(3, R=1.1, jitter=0.2, seed=7)
    s, lk = _fields(m, 31)
    _, N = oracle.dofs(m)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((2, N))
    L = rng.standard_normal((2, N))
    g2 = oracle.grad(m, s, lk, U, L, s_bar=SBAR, n_sing=NS)
    g0 = oracle.grad(m, s, lk, U[0], L[0], s_bar=SBAR, n_sing=NS)
    g1 = oracle.grad(m, s, lk, U[1], L[1], s_bar=SBAR, n_sing=NS)
    for a, b, c in zip(g2, g0, g1):
        np.testing.assert_allclose(a, b + c, rtol=1e-12, atol=1e-12 * np.abs(a).max())


def test_grad_rejects_analytic_or_tail():
    m = synth.disk_mesh(3, R=1.1, jitter=0.2, seed=5)
    with pytest.raises(ValueError):
        oracle.grad(m, np.full(m.n_vert, 0.5), np.zeros(m.n_vert), np.zeros(3), np.zeros(3))
