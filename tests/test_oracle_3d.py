"""Pins of the oracle's 3D (tetrahedral) separated parts on small Kuhn-grid
balls: K (eq. e:k), the density rho by the direct point sum (Sec. 6.1) and the
weighted mass M (eq. e:m), with the symmetric 4-point degree-2 element rule
(reading R20; the paper gives no singular rules for tetrahedron pairs, so B is
not assembled in 3D).

* gamma == 1 (s = -3/2, kappa = 1): rho(q) = |Omega| - |S_tau|, K_ij =
  -2 sum over separated interior pairs of (|tau|/4)(|tau'|/4), and M_ij =
  2 sum_tau rho_tau |tau| (1 + delta_ab)/20 (exact only if the rule integrates
  quadratics exactly) -- closed forms;
* a variable kernel (s = 0.3, a 3D Fourier log kappa) against a numpy brute
  force of the same sums written from the definitions;
* single-row applies (rows of K + M) and the P1 load in 3D; refusals of what
  needs singular rules or the 2D tail.
"""
import math

import numpy as np
import pytest

import oracle
import synth

RA, RB = (5 + 3 * math.sqrt(5)) / 20, (5 - math.sqrt(5)) / 20   # 4-point rule (R20)


def _vol(m):
    P = m.coords[m.cells]
    return np.abs(np.einsum("ij,ij->i", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6


def _touch(m):
    """(C x C) bool: cells sharing at least one vertex (a cell touches itself)."""
    inc = np.zeros((m.n_cell, m.n_vert))
    inc[np.repeat(np.arange(m.n_cell), 4), m.cells.ravel()] = 1.0
    return (inc @ inc.T) > 0


@pytest.fixture(scope="module")
def ball():
    m = synth.kuhn_ball_mesh(5)
    assert m.d == 3 and m.n_cell > 300
    return m


def test_gamma_one_closed_forms(ball):
    m = ball
    ref = oracle.assemble(m, synth.const_field(-1.5), synth.const_field(0.0), s_bar=0.9)
    vol, T = _vol(m), _touch(m)
    dof, N = oracle.dofs(m)
    inter = np.nonzero(m.cell_is_interior)[0]
    total = vol.sum()
    rho_c = total - T[inter] @ vol                       # per interior cell
    assert np.abs(ref.rho - np.repeat(rho_c, 4)).max() <= 1e-12 * total
    # K = -2 E^T W E, E_c = (|tau|/4) on the DoFs of c, W = separated interior pairs
    E = np.zeros((len(inter), N))
    for r, c in enumerate(inter):
        for v in m.cells[c]:
            if dof[v] >= 0:
                E[r, dof[v]] += vol[c] / 4
    W = ~T[np.ix_(inter, inter)]
    K = -2.0 * E.T @ W @ E
    scale = np.abs(K).max()
    assert scale > 0 and np.abs(ref.K - K).max() <= 1e-12 * scale
    Mref = np.zeros((N, N))
    for r, c in enumerate(inter):
        for a, va in enumerate(m.cells[c]):
            for b, vb in enumerate(m.cells[c]):
                if dof[va] >= 0 and dof[vb] >= 0:
                    Mref[dof[va], dof[vb]] += 2.0 * rho_c[r] * vol[c] * (2.0 if a == b else 1.0) / 20
    assert np.abs(ref.M - Mref).max() <= 1e-12 * np.abs(Mref).max()
    assert not ref.B.any()


def _fourier(f, x):
    v = np.full(len(x), float(f.c0))
    for row in np.asarray(f.fourier, dtype=float).reshape(-1, 5):
        v += row[3] * np.cos(math.pi * (x @ row[:3]) + row[4])
    return v


def test_variable_kernel_brute_force():
    m = synth.kuhn_ball_mesh(4)
    s0 = 0.3
    fk = synth.random_fourier_field(7, 0.5, d=3)
    ref = oracle.assemble(m, synth.const_field(s0), fk, s_bar=0.9)
    vol, T = _vol(m), _touch(m)
    dof, N = oracle.dofs(m)
    lam = np.full((4, 4), RB) + (RA - RB) * np.eye(4)     # lam[q][a]
    P = m.coords[m.cells]                                 # C x 4 x 3
    xq = np.einsum("qa,cai->cqi", lam, P).reshape(-1, 3)  # points cell-major
    wq = np.repeat(vol / 4, 4)
    lk = _fourier(fk, xq)
    cell_of = np.repeat(np.arange(m.n_cell), 4)
    sep = ~T[np.ix_(cell_of, cell_of)]
    r = np.linalg.norm(xq[:, None, :] - xq[None, :, :], axis=2)
    with np.errstate(divide="ignore"):
        G = np.where(sep, np.exp(0.5 * (lk[:, None] + lk[None, :])) * r ** -(3 + 2 * s0), 0.0)
    inter_pts = np.nonzero(np.repeat(m.cell_is_interior, 4))[0]
    rho = G[inter_pts] @ wq
    assert np.abs(ref.rho - rho).max() <= 1e-12 * np.abs(rho).max()
    # K_ij = -2 sum over interior points of w w' psi_i psi_j gamma (separated)
    Psi = np.zeros((len(xq), N))
    for c in range(m.n_cell):
        if not m.cell_is_interior[c]:
            continue
        for a, v in enumerate(m.cells[c]):
            if dof[v] >= 0:
                Psi[4 * c:4 * c + 4, dof[v]] = lam[:, a]
    K = -2.0 * (Psi * wq[:, None]).T @ G @ (Psi * wq[:, None])
    assert np.abs(ref.K - K).max() <= 1e-12 * np.abs(K).max()
    assert np.allclose(ref.K, ref.K.T, rtol=0, atol=1e-14 * np.abs(K).max())
    assert np.allclose(ref.M, ref.M.T, rtol=0, atol=1e-14 * np.abs(ref.M).max())


def test_load_3d(ball):
    m = ball
    vol = _vol(m)
    dof, N = oracle.dofs(m)
    F1 = oracle.load(m, np.ones(m.n_vert))
    Fx = oracle.load(m, m.coords[:, 0].copy())
    e1, ex = np.zeros(N), np.zeros(N)
    for c in np.nonzero(m.cell_is_interior)[0]:
        for a, va in enumerate(m.cells[c]):
            if dof[va] < 0:
                continue
            e1[dof[va]] += vol[c] / 4                     # int psi_i
            for b, vb in enumerate(m.cells[c]):           # int psi_i x, x linear
                ex[dof[va]] += vol[c] * (2.0 if a == b else 1.0) / 20 * m.coords[vb, 0]
    assert np.abs(F1 - e1).max() <= 1e-13 * e1.max()
    assert np.abs(Fx - ex).max() <= 1e-13 * e1.max()


def test_single_rows_3d(ball):
    """oracle.apply_rows in 3D gives the rows of K + M (B = 0) of the dense assembly."""
    m = ball
    s, k = synth.const_field(0.4), synth.random_fourier_field(11, 0.5, d=3)
    ref = oracle.assemble(m, s, k, s_bar=0.9)
    x = np.random.default_rng(5).standard_normal(ref.N)
    rows = np.arange(0, ref.N, 3)
    y = oracle.apply_rows(m, s, k, x, rows, s_bar=0.9)
    yd = (ref.K + ref.M) @ x
    assert np.abs(y - yd[rows]).max() <= 1e-12 * np.abs(yd).max()


def test_3d_refuses_what_needs_singular_rules(ball):
    s, k = synth.const_field(0.3), synth.const_field(0.0)
    with pytest.raises(RuntimeError):
        oracle.assemble(ball, s, k, want_full=True)
    with pytest.raises(RuntimeError):
        oracle.assemble(ball, s, k, tail=1)
    with pytest.raises(ValueError):
        oracle.apply_rows(ball, s, k, np.zeros(oracle.dofs(ball)[1]), [0], tail=1)
