"""The 3D (tetrahedral) GPU path against the oracle's 3D separated parts: the
operator K + M of Sec. 3 on Kuhn-grid balls (the 4-point element rule of
reading R20; B = 0, since the paper gives no singular rules for tetrahedron
pairs), with the 3D configuration's fields (Gaussian-bump order, 3D Fourier
log kappa).

* exact mode (every block near, direct density): the GPU matrix equals the
  oracle's dense K + M to 1e-11, and the FP64 CG solution its Cholesky
  solution to 1e-8;
* H^2 mode (lambda 0.75, Chebyshev p = 4, rank 64): sampled exact rows of
  A x, and the matvec error falls with the interpolation order;
* the P1 load vector; the mixed-precision solve (FP32 coupling, FP64
  residuals, 16 right-hand sides) reaches the FP64 solution.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


@pytest.fixture(scope="module")
def ball():
    m, s, k, prm = synth.ball_workload(8)
    ref = oracle.assemble(m, s, k, s_bar=0.9)
    return m, s, k, prm, ref


def _map(mesh, ref):
    dof, n = vfd.vfd_mesh_dofs(mesh)
    assert n == ref.N
    sel = dof >= 0
    return dof[sel], ref.dof[sel]


def test_3d_exact_mode_matrix_and_solve(ball):
    m, s, k, prm, ref = ball
    mesh = vfd.vfd_mesh(3, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=0.0, rho_lambda=0.0)
    gi, oi = _map(mesh, ref)
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    A = ref.K + ref.M
    rng = np.random.default_rng(1)
    n = ref.N
    for _ in range(2):
        xo = rng.standard_normal(n)
        xg = np.zeros(n)
        xg[gi] = xo[oi]
        X = torch.tensor(xg, device="cuda")
        Y = torch.empty_like(X)
        vfd.vfd_apply(op, X, Y)
        torch.cuda.synchronize()
        yo = A @ xo
        assert np.abs(Y.cpu().numpy()[gi] - yo[oi]).max() / np.abs(yo).max() < 1e-11
    Fo = oracle.load(m, np.ones(m.n_vert))
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device="cuda"), F)
    torch.cuda.synchronize()
    assert np.abs(F.cpu().numpy()[gi] - Fo[oi]).max() <= 1e-13 * np.abs(Fo).max()
    U = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(op, F, U, rtol=1e-13, max_it=10000)
    Uo = oracle.cholesky_solve(A, Fo)
    assert np.linalg.norm(U.cpu().numpy()[gi] - Uo[oi]) / np.linalg.norm(Uo) < 1e-8


@pytest.mark.parametrize("p,tol", [(3, 2e-3), (4, 5e-4)])
def test_3d_h2_rows(ball, p, tol):
    m, s, k, prm, ref = ball
    mesh = vfd.vfd_mesh(3, m.coords, m.cells, m.cell_is_interior, leaf_m=32, cheb_p=p, lam=0.75, rho_lambda=0.75)
    assert mesh.info["rank"] == p ** 3
    gi, oi = _map(mesh, ref)
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    xo = np.random.default_rng(2).standard_normal(ref.N)
    xg = np.zeros(ref.N)
    xg[gi] = xo[oi]
    X = torch.tensor(xg, device="cuda")
    Y = torch.empty_like(X)
    vfd.vfd_apply(op, X, Y)
    torch.cuda.synchronize()
    yo = (ref.K + ref.M) @ xo
    err = np.abs(Y.cpu().numpy()[gi] - yo[oi]).max() / np.abs(yo).max()
    print(f"3D H^2 p={p}: {err:.2e}, far blocks {mesh.info['far_blocks']}")
    assert err < tol


def test_3d_mixed_precision_16_rhs(ball):
    m, s, k, prm, ref = ball
    mesh = vfd.vfd_mesh(3, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=0.75, rho_lambda=0.75)
    n = mesh.n_dof
    op64 = vfd.vfd_assemble(mesh, s, k, 0.9)
    op32 = vfd.vfd_assemble(mesh, s, k, 0.9, precision=vfd.VFD_FP32)
    g = torch.Generator(device="cuda").manual_seed(9)
    F = torch.randn(16, n, dtype=torch.float64, device="cuda", generator=g)
    U64 = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(op64, F, U64, rtol=1e-11, max_it=20000)
    assert st == vfd.VFD_OK
    U = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(op32, F, U, rtol=1e-8, max_it=20000)
    assert st == vfd.VFD_OK and np.all(rel <= 1e-8)
    d = (torch.linalg.norm(U - U64, dim=1) / torch.linalg.norm(U64, dim=1)).max().item()
    assert d < 1e-6, d


def test_3d_full_size_rows():
    """A larger ball (24^3 grid, about 5k DoFs) in the configuration's mesh
    options (leaf 64, p = 4): sampled exact rows of A x from the oracle."""
    m, s, k, prm = synth.ball_workload(24)
    mesh = vfd.vfd_mesh(3, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], cheb_p=prm["p"],
                        lam=prm["lam"], rho_lambda=prm["lam"])
    op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"])
    dof_o, N = oracle.dofs(m)
    dof, n = vfd.vfd_mesh_dofs(mesh)
    assert n == N
    rng = np.random.default_rng(4)
    xv = rng.standard_normal(m.n_vert)
    sel = np.nonzero(dof >= 0)[0]
    xg = np.zeros(n)
    xg[dof[sel]] = xv[sel]
    xo = np.zeros(N)
    xo[dof_o[sel]] = xv[sel]
    X = torch.tensor(xg, device="cuda")
    Y = torch.empty_like(X)
    vfd.vfd_apply(op, X, Y)
    torch.cuda.synchronize()
    verts = rng.choice(sel, 16, replace=False)
    yo = oracle.apply_rows(m, s, k, xo, dof_o[verts], s_bar=prm["s_bar"])
    yg = Y.cpu().numpy()[dof[verts]]
    err = np.abs(yg - yo).max() / np.abs(yo).max()
    print(f"3D 24^3 ball, {n} DoFs: sampled-row error {err:.2e}")
    assert err < 1e-3
