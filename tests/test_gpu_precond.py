"""Two-level preconditioned CG (vfd_precondition) on the GPU.

The preconditioner changes the iteration, not the system: the PCG solution
must match the oracle's dense Cholesky solve (exact mode) and the plain-CG
solution of the same H^2 operator, with fewer iterations.  VFD_PREC_NONE
restores plain CG (same iteration count as before); low-precision operators
and unknown kinds are rejected.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


def _rhs(mesh, n_vert, n):
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    vfd.vfd_load(mesh, torch.ones(n_vert, dtype=torch.float64, device="cuda"), F)
    return F


def test_pcg_matches_oracle_exact_mode():
    m = synth.disk_mesh(7, R=1.3, jitter=0.2, seed=11)
    s = synth.config2_s_field()
    k = synth.random_fourier_field(21, 0.5)
    ref = oracle.assemble(m, s, k, s_bar=0.9, n_sing=3)
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=16, lam=0.0, rho_lambda=0.0)
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    dof, n = vfd.vfd_mesh_dofs(mesh)
    sel = dof >= 0
    gi, oi = dof[sel], ref.dof[sel]
    U_or = oracle.cholesky_solve(ref.A, oracle.load(m, np.ones(m.n_vert)))
    F = _rhs(mesh, m.n_vert, n)
    U0 = torch.zeros_like(F)
    st, it0, _ = vfd.vfd_solve(op, F, U0, rtol=1e-12, max_it=5000)
    assert st == vfd.VFD_OK
    vfd.vfd_precondition(op)
    U1 = torch.zeros_like(F)
    st, it1, rel = vfd.vfd_solve(op, F, U1, rtol=1e-12, max_it=5000)
    assert st == vfd.VFD_OK and rel[0] <= 1e-12
    Ug = U1.cpu().numpy()
    assert np.linalg.norm(Ug[gi] - U_or[oi]) / np.linalg.norm(U_or) < 1e-8
    assert it1[0] < it0[0], (it0, it1)


@pytest.fixture(scope="module")
def h2_case():
    m = synth.disk_mesh_for_dofs(12000, R=1.1, jitter=0.2, seed=3)
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=32, cheb_p=6, lam=0.75, rho_leaf_m=64,
                        rho_lambda=0.75)
    s = synth.config2_s_field()
    k = synth.random_fourier_field(21, 0.5)
    return m, mesh, s, k


def test_pcg_h2_operator_same_solution_fewer_iterations(h2_case):
    m, mesh, s, k = h2_case
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    n = mesh.n_dof
    rng = np.random.default_rng(7)
    F = torch.tensor(rng.standard_normal((3, n)), device="cuda")
    U0 = torch.zeros_like(F)
    st, it0, _ = vfd.vfd_solve(op, F, U0, rtol=1e-10, max_it=20000)
    assert st == vfd.VFD_OK
    vfd.vfd_precondition(op, vfd.VFD_PREC_TWO_LEVEL)
    U1 = torch.zeros_like(F)
    st, it1, rel = vfd.vfd_solve(op, F, U1, rtol=1e-10, max_it=20000)
    assert st == vfd.VFD_OK and max(rel) <= 1e-10
    for r in range(3):
        err = (torch.linalg.norm(U1[r] - U0[r]) / torch.linalg.norm(U0[r])).item()
        assert err < 1e-7, (r, err)
        assert it1[r] < it0[r], (it0, it1)
    # the true residual of the PCG solution
    Y = torch.empty_like(U1)
    vfd.vfd_apply(op, U1, Y)
    res = (torch.linalg.norm(F - Y, dim=1) / torch.linalg.norm(F, dim=1)).max().item()
    assert res < 1e-9, res
    # back to plain CG: the iteration counts of the first solve
    vfd.vfd_precondition(op, vfd.VFD_PREC_NONE)
    U2 = torch.zeros_like(F)
    st, it2, _ = vfd.vfd_solve(op, F, U2, rtol=1e-10, max_it=20000)
    assert st == vfd.VFD_OK and list(it2) == list(it0)


def test_precondition_rejects_lowp_and_unknown_kind(h2_case):
    m, mesh, s, k = h2_case
    op32 = vfd.vfd_assemble(mesh, s, k, 0.9, precision=vfd.VFD_FP32)
    with pytest.raises(vfd.VfdError) as e:
        vfd.vfd_precondition(op32)
    assert e.value.status == vfd.VFD_EUNSUPPORTED
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    with pytest.raises(vfd.VfdError) as e:
        vfd.vfd_precondition(op, 7)
    assert e.value.status == vfd.VFD_EINVAL
