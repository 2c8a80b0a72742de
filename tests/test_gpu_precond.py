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


def test_block_jacobi_between_none_and_two_level(h2_case):
    m, mesh, s, k = h2_case
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    F = _rhs(mesh, m.n_vert, mesh.n_dof)
    its, sols = {}, {}
    for kind in (vfd.VFD_PREC_NONE, vfd.VFD_PREC_BLOCK_JACOBI, vfd.VFD_PREC_TWO_LEVEL):
        vfd.vfd_precondition(op, kind)
        U = torch.zeros_like(F)
        st, it, _ = vfd.vfd_solve(op, F, U, rtol=1e-10, max_it=20000)
        assert st == vfd.VFD_OK
        its[kind], sols[kind] = it[0], U
    print("iterations none / block Jacobi / two-level:", its)
    assert its[vfd.VFD_PREC_TWO_LEVEL] < its[vfd.VFD_PREC_BLOCK_JACOBI] < its[vfd.VFD_PREC_NONE]
    for kind in (vfd.VFD_PREC_BLOCK_JACOBI, vfd.VFD_PREC_TWO_LEVEL):
        err = (torch.linalg.norm(sols[kind] - sols[0]) / torch.linalg.norm(sols[0])).item()
        assert err < 1e-7, (kind, err)


def test_precondition_unknown_kind(h2_case):
    m, mesh, s, k = h2_case
    op = vfd.vfd_assemble(mesh, s, k, 0.9)
    with pytest.raises(vfd.VfdError) as e:
        vfd.vfd_precondition(op, 7)
    assert e.value.status == vfd.VFD_EINVAL


@pytest.mark.parametrize("prec", [vfd.VFD_FP32, vfd.VFD_BF16])
def test_batched_mixed_precision_pcg(h2_case, prec):
    """64 right-hand sides on a low-precision operator: the preconditioned
    batched solve (FP32 copies of the inverses, reliable updates with the FP64
    operator) reaches the same solution as the FP64 CG with far fewer inner
    iterations than the unpreconditioned batched solve."""
    m, mesh, s, k = h2_case
    op64 = vfd.vfd_assemble(mesh, s, k, 0.9)
    opl = vfd.vfd_assemble(mesh, s, k, 0.9, precision=prec)
    n = mesh.n_dof
    gen = torch.Generator(device="cuda").manual_seed(17)
    F = torch.randn(64, n, dtype=torch.float64, device="cuda", generator=gen)
    vfd.vfd_precondition(op64)
    U64 = torch.zeros_like(F)
    st, _, _ = vfd.vfd_solve(op64, F, U64, rtol=1e-11, max_it=20000)
    assert st == vfd.VFD_OK
    U0 = torch.zeros_like(F)
    st, it0, _ = vfd.vfd_solve(opl, F, U0, rtol=1e-8, max_it=20000)
    assert st == vfd.VFD_OK
    vfd.vfd_precondition(opl)
    U1 = torch.zeros_like(F)
    st, it1, rel = vfd.vfd_solve(opl, F, U1, rtol=1e-8, max_it=20000)
    print(f"batched inner iterations: plain {it0.max()}, preconditioned {it1.max()}")
    assert st == vfd.VFD_OK and rel.max() <= 1e-8
    err = (torch.linalg.norm(U1 - U64, dim=1) / torch.linalg.norm(U64, dim=1)).max().item()
    assert err < 1e-6, err
    assert it1.max() * 3 < it0.max(), (it0.max(), it1.max())
    # back to plain
    vfd.vfd_precondition(opl, vfd.VFD_PREC_NONE)
    U2 = torch.zeros_like(F)
    st, it2, _ = vfd.vfd_solve(opl, F, U2, rtol=1e-8, max_it=20000)
    assert st == vfd.VFD_OK and it2.max() == it0.max()


def test_batch_of_meshes_pcg_matches_single_solves():
    """Three meshes of different sizes in one preconditioned batched solve:
    each mesh's solution equals its own FP64 solve; preconditioning only part
    of a batch is rejected."""
    meshes = [synth.disk_mesh_for_dofs(n, seed=40 + i) for i, n in enumerate((1500, 4000, 9000))]
    s = synth.config2_s_field()
    k = synth.random_fourier_field(21, 0.5)
    ops, ops64, Fs, Us, refs = [], [], [], [], []
    for i, mm in enumerate(meshes):
        mesh = vfd.vfd_mesh(2, mm.coords, mm.cells, mm.cell_is_interior, leaf_m=32, lam=0.75, rho_lambda=0.75)
        op = vfd.vfd_assemble(mesh, s, k, 0.9, precision=vfd.VFD_FP32)
        op64 = vfd.vfd_assemble(mesh, s, k, 0.9)
        gen = torch.Generator(device="cuda").manual_seed(60 + i)
        F = torch.randn(64, mesh.n_dof, dtype=torch.float64, device="cuda", generator=gen)
        U = torch.zeros_like(F)
        vfd.vfd_precondition(op64)
        st, _, _ = vfd.vfd_solve(op64, F, U, rtol=1e-11, max_it=20000)
        assert st == vfd.VFD_OK
        ops.append(op)
        ops64.append(op64)
        Fs.append(F)
        Us.append(torch.zeros_like(F))
        refs.append(U)
    vfd.vfd_precondition(ops[0])
    batch = vfd.vfd_batch_create(ops)
    with pytest.raises(vfd.VfdError) as e:
        vfd.vfd_batch_solve(batch, Fs, Us, rtol=1e-8)
    assert e.value.status == vfd.VFD_EINVAL
    for op in ops[1:]:
        vfd.vfd_precondition(op)
    st, it, rel = vfd.vfd_batch_solve(batch, Fs, Us, rtol=1e-8)
    assert st == vfd.VFD_OK and rel.max() <= 1e-8
    for U, ref in zip(Us, refs):
        err = (torch.linalg.norm(U - ref, dim=1) / torch.linalg.norm(ref, dim=1)).max().item()
        assert err < 1e-6, err
