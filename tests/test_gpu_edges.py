"""Edge cases through the C ABI: degenerate meshes, ragged column counts,
zero right-hand sides, several 64-column tiles, a single leaf.

* a mesh whose cells are all exterior has no DoFs: setup reports n_dof = 0 and
  the operator's calls are no-ops or clean errors;
* a one-leaf K tree (leaf size >= DoFs) has no low-rank blocks at any lambda
  and, with the direct density, matches the oracle;
* zero right-hand sides: the solvers return U = 0 with zero iterations;
* 65 columns (ragged: one full 64-column tile plus one column in the padded
  batched solve) and 128 columns (two RHS tiles per CTA grid) through the
  batched path, against the FP64 operator.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


def _fields():
    return synth.config2_s_field(), synth.random_fourier_field(31, 0.5)


def test_no_interior_dofs():
    m = synth.disk_mesh(4, R=1.1, jitter=0.2, seed=1)
    inter = np.zeros_like(m.cell_is_interior)
    try:
        mesh = vfd.vfd_mesh(2, m.coords, m.cells, inter, leaf_m=16, lam=0.0, rho_lambda=0.0)
    except vfd.VfdError as e:   # refusing an empty problem is also acceptable, with a clear status
        assert e.status == vfd.VFD_EINVAL
        return
    assert mesh.n_dof == 0


def test_single_leaf_matches_oracle():
    m = synth.disk_mesh(5, R=1.1, jitter=0.2, seed=2)
    s, k = _fields()
    ref = oracle.assemble(m, s, k, s_bar=0.9, n_sing=3)
    # K: one leaf, so no admissible block even at lambda = 0.75; the density direct (rho_lambda = 0)
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=256, lam=0.75, rho_lambda=0.0)
    assert mesh.info["far_blocks"] == 0
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    dof, n = vfd.vfd_mesh_dofs(mesh)
    sel = dof >= 0
    x = np.random.default_rng(3).standard_normal(n)
    X = torch.tensor(x, device="cuda")
    Y = torch.empty_like(X)
    vfd.vfd_apply(op, X, Y)
    torch.cuda.synchronize()
    xo = np.zeros(ref.N)
    xo[ref.dof[sel]] = x[dof[sel]]
    yo = ref.A @ xo
    err = np.abs(Y.cpu().numpy()[dof[sel]] - yo[ref.dof[sel]]).max() / np.abs(yo).max()
    assert err < 1e-11, err


@pytest.mark.parametrize("prec,nrhs", [(vfd.VFD_FP64, 1), (vfd.VFD_FP64, 3), (vfd.VFD_FP32, 1), (vfd.VFD_BF16, 64)])
def test_zero_rhs(prec, nrhs):
    m = synth.disk_mesh(8, R=1.1, jitter=0.2, seed=3)
    s, k = _fields()
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=0.75, rho_lambda=0.75)
    op = vfd.vfd_assemble(mesh, s, k, 0.9, precision=prec)
    shape = (mesh.n_dof,) if nrhs == 1 else (nrhs, mesh.n_dof)
    F = torch.zeros(*shape, dtype=torch.float64, device="cuda")
    U = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(op, F, U, rtol=1e-10, max_it=1000)
    assert st == vfd.VFD_OK
    assert torch.count_nonzero(U).item() == 0
    assert np.all(it == 0)


@pytest.mark.parametrize("nrhs", [65, 128])
def test_ragged_and_multi_tile_columns(nrhs):
    m = synth.disk_mesh(14, R=1.1, jitter=0.2, seed=9)
    s, k = _fields()
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=0.75, rho_lambda=0.75)
    op64 = vfd.vfd_assemble(mesh, s, k, 0.9)
    op32 = vfd.vfd_assemble(mesh, s, k, 0.9, precision=vfd.VFD_FP32)
    g = torch.Generator(device="cuda").manual_seed(nrhs)
    X = torch.randn(nrhs, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    Y64 = torch.empty_like(X)
    Y32 = torch.empty_like(X)
    vfd.vfd_apply(op64, X, Y64)
    vfd.vfd_apply(op32, X, Y32)   # 128: batched path with two RHS tiles; 65: column path
    torch.cuda.synchronize()
    err = (torch.linalg.norm(Y32 - Y64, dim=1) / torch.linalg.norm(Y64, dim=1)).max().item()
    assert err < 2e-3, err
    # the batched refinement pads the columns to a multiple of 64
    F = X.clone()
    F[3].zero_()   # one column converged from the start
    U = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(op32, F, U, rtol=1e-9, max_it=50000)
    assert st == vfd.VFD_OK and rel.max() <= 1e-9
    assert torch.count_nonzero(U[3]).item() == 0
    AU = torch.empty_like(U)
    vfd.vfd_apply(op64, U, AU)
    torch.cuda.synchronize()
    live = [c for c in range(nrhs) if c != 3]
    r = (torch.linalg.norm(F[live] - AU[live], dim=1) / torch.linalg.norm(F[live], dim=1)).max().item()
    assert r <= 1.01e-9, r
