"""Graded exterior meshes on the GPU path (the remark of Sec. 7.2): the graded
square (interior as the quasi-uniform square, exterior cells growing
geometrically) through the C ABI against the oracle's dense assembly -- the
exact-mode operator (every block near, direct density) to 1e-11, its solve
against the oracle's Cholesky solution to 1e-8 -- and the H^2 operator's
density needs fewer source points than the quasi-uniform exterior's."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


def test_graded_square_exact_parity():
    m = synth.square_mesh_graded(16, 1.5)
    s = synth.config2_s_field()
    k = synth.random_fourier_field(61, 0.5)
    ref = oracle.assemble(m, s, k, s_bar=0.9, n_sing=3)
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=0.0, rho_lambda=0.0)
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    dof, n = vfd.vfd_mesh_dofs(mesh)
    assert n == ref.N
    sel = dof >= 0
    gi, oi = dof[sel], ref.dof[sel]
    rng = np.random.default_rng(3)
    xo = rng.standard_normal(n)
    xg = np.zeros(n)
    xg[gi] = xo[oi]
    X = torch.tensor(xg, device="cuda")
    Y = torch.empty_like(X)
    vfd.vfd_apply(op, X, Y)
    torch.cuda.synchronize()
    yo = ref.A @ xo
    yg = Y.cpu().numpy()
    assert np.abs(yg[gi] - yo[oi]).max() / np.abs(yo).max() < 1e-11
    F = torch.ones(n, dtype=torch.float64, device="cuda")
    U = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(op, F, U, rtol=1e-13, max_it=5000)
    Uo = oracle.cholesky_solve(ref.A, np.ones(n))
    ug = U.cpu().numpy()
    assert np.linalg.norm(ug[gi] - Uo[oi]) / np.linalg.norm(Uo) < 1e-8


def test_graded_square_density_sources():
    mu = synth.square_mesh(32)
    mg = synth.square_mesh_graded(32, 1.5)
    iu = vfd.vfd_mesh(2, mu.coords, mu.cells, mu.cell_is_interior).info
    ig = vfd.vfd_mesh(2, mg.coords, mg.cells, mg.cell_is_interior).info
    assert ig["n_dof"] == iu["n_dof"] and ig["n_qint"] == iu["n_qint"]
    assert ig["n_q"] < 0.55 * iu["n_q"]
