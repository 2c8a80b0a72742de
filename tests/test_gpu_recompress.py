"""Algebraic recompression of the far field (mesh option recompress_tol, the
last paragraph of Sec. 5.3): per-node orthogonalised bases cut to the
singular directions of their coupling rows.

* the recompressed operator against the interpolation operator it was cut
  from (same mesh, fields): relative matvec error within a small multiple of
  the tolerance, and against the oracle's dense matrix within the H^2
  interpolation tolerance;
* the per-level ranks fall below the interpolation rank and shrink with a
  looser tolerance;
* the no-allocation apply equals the apply on the recompressed operator;
* FP64 CG and the 64-RHS mixed-precision solve reach the solution of the
  interpolation operator to the recompression level.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402

SBAR = 0.9


@pytest.fixture(scope="module")
def disk():
    m = synth.disk_mesh(14, R=1.1, jitter=0.2, seed=14)
    s = synth.config2_s_field()
    k = synth.random_fourier_field(21, 0.5)
    ref = oracle.assemble(m, s, k, s_bar=SBAR, n_sing=3)
    return m, s, k, ref


def _mesh(m, tol, p=8, lam=0.5, leaf=16):
    return vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=leaf, cheb_p=p, lam=lam, rho_leaf_m=32,
                        rho_lambda=lam, recompress_tol=tol)


def _apply(op, X):
    Y = torch.empty_like(X)
    vfd.vfd_apply(op, X, Y)
    return Y


@pytest.mark.parametrize("tol", [1e-10, 1e-8, 1e-6])
def test_recompressed_apply(disk, tol):
    m, s, k, ref = disk
    mesh0, mesh = _mesh(m, 0.0), _mesh(m, tol)
    op0 = vfd.vfd_assemble(mesh0, s, k, SBAR)
    op = vfd.vfd_assemble(mesh, s, k, SBAR)
    ranks = vfd.vfd_op_far_ranks(op)
    assert len(ranks) > 0 and all(r <= 64 for r in ranks) and min(ranks) < 64, ranks
    g = torch.Generator(device="cuda").manual_seed(3)
    X = torch.randn(3, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    Y0, Y = _apply(op0, X), _apply(op, X)
    err = (torch.linalg.norm(Y - Y0) / torch.linalg.norm(Y0)).item()
    # against the dense oracle matrix
    dof, n = vfd.vfd_mesh_dofs(mesh)
    sel = dof >= 0
    gi, oi = dof[sel], ref.dof[sel]
    xo = np.zeros(ref.N)
    xo[oi] = X[0].cpu().numpy()[gi]
    yo = ref.A @ xo
    err_o = np.linalg.norm(Y[0].cpu().numpy()[gi] - yo[oi]) / np.linalg.norm(yo)
    print(f"tol {tol:.0e}: ranks {ranks}, vs interpolation operator {err:.2e}, vs oracle {err_o:.2e}")
    assert err < 30 * tol, err
    assert err_o < 2e-5 + 30 * tol, err_o


def test_ranks_shrink_with_tolerance(disk):
    m, s, k, _ = disk
    r = {}
    for tol in (1e-10, 1e-6):
        op = vfd.vfd_assemble(_mesh(m, tol), s, k, SBAR)
        r[tol] = vfd.vfd_op_far_ranks(op)
    assert all(a >= b for a, b in zip(r[1e-10], r[1e-6])) and sum(r[1e-6]) < sum(r[1e-10]), r


def test_noalloc_equals_apply_recompressed(disk):
    m, s, k, _ = disk
    op = vfd.vfd_assemble(_mesh(m, 1e-9), s, k, SBAR)
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(2, op.mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    Y = _apply(op, X)
    Yn = torch.empty_like(X)
    vfd.vfd_apply_noalloc(op, X, Yn)
    torch.cuda.synchronize()
    assert torch.equal(Y, Yn)


def test_solves_with_recompression(disk):
    m, s, k, _ = disk
    mesh0, mesh = _mesh(m, 0.0, leaf=32), _mesh(m, 1e-10, leaf=32)
    op0 = vfd.vfd_assemble(mesh0, s, k, SBAR)
    g = torch.Generator(device="cuda").manual_seed(7)
    F = torch.randn(64, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    U0 = torch.zeros_like(F)
    st, _, _ = vfd.vfd_solve(op0, F[:2], U0[:2], rtol=1e-11, max_it=20000)
    assert st == vfd.VFD_OK
    op = vfd.vfd_assemble(mesh, s, k, SBAR)
    U1 = torch.zeros_like(F)
    st, _, _ = vfd.vfd_solve(op, F[:2], U1[:2], rtol=1e-11, max_it=20000)
    assert st == vfd.VFD_OK
    e64 = (torch.linalg.norm(U1[:2] - U0[:2], dim=1) / torch.linalg.norm(U0[:2], dim=1)).max().item()
    # 64 columns through the batched mixed-precision solve (FP64 residuals of the recompressed operator)
    opl = vfd.vfd_assemble(mesh, s, k, SBAR, precision=vfd.VFD_FP32)
    U2 = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(opl, F, U2, rtol=1e-9, max_it=20000)
    assert st == vfd.VFD_OK
    emx = (torch.linalg.norm(U2[:2] - U0[:2], dim=1) / torch.linalg.norm(U0[:2], dim=1)).max().item()
    print(f"solution vs interpolation operator: FP64 CG {e64:.2e}, mixed 64-RHS {emx:.2e}")
    assert e64 < 1e-7 and emx < 1e-6, (e64, emx)
