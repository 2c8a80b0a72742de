"""Failure reporting of the solvers, made on the host side (no GPU fault):
every solver given far too few iterations returns VFD_ENOCONV, leaves its
last iterate in U (finite, with a lower energy U.AU/2 - F.U than the initial
guess) and reports the residual it reached.  Covers the FP64 CG (Sec. 7), the
single-column iterative refinement of VFD_FP32 and VFD_BF16 operators, the
64-column mixed-precision solve of one operator and the batched solve over
several meshes.  Also: a VFD_BF16 operator applied column by column equals
the VFD_FP32 operator (both use FP32 copies of K off the batched path).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    m = synth.disk_mesh(16, R=1.1, jitter=0.2, seed=41)
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=0.75, rho_lambda=0.75)
    s = synth.config2_s_field()
    k = synth.random_fourier_field(42, 0.5)
    ops = {p: vfd.vfd_assemble(mesh, s, k, 0.9, precision=p) for p in (vfd.VFD_FP64, vfd.VFD_FP32, vfd.VFD_BF16)}
    F = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device="cuda"), F)
    return m, mesh, ops, F


@pytest.mark.parametrize("prec", [vfd.VFD_FP64, vfd.VFD_FP32, vfd.VFD_BF16])
def test_single_column_noconv_keeps_last_iterate(setup, prec):
    m, mesh, ops, F = setup
    U = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(ops[prec], F, U, rtol=1e-12, max_it=3)
    assert st == vfd.VFD_ENOCONV
    assert int(it[0]) <= 3
    assert torch.isfinite(U).all().item() and torch.count_nonzero(U).item() > 0
    # CG decreases the energy J(U) = U.AU/2 - F.U (J(0) = 0) even when the
    # residual norm grows in the first iterations
    AU = torch.empty_like(U)
    vfd.vfd_apply(ops[vfd.VFD_FP64], U, AU)
    torch.cuda.synchronize()
    assert (0.5 * (U @ AU) - F @ U).item() < 0.0
    r = (torch.linalg.norm(F - AU) / torch.linalg.norm(F)).item()
    assert abs(r - rel[0]) <= 1e-6 * r     # the reported residual is the true one of the returned U
    assert rel[0] > 1e-12
    # the same call with enough iterations converges
    U.zero_()
    st, it, rel = vfd.vfd_solve(ops[prec], F, U, rtol=1e-10, max_it=100000)
    assert st == vfd.VFD_OK and rel[0] <= 1e-10


def test_multi_column_noconv(setup):
    m, mesh, ops, F = setup
    g = torch.Generator(device="cuda").manual_seed(3)
    Fb = torch.randn(64, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    for prec in (vfd.VFD_FP32, vfd.VFD_BF16):
        U = torch.zeros_like(Fb)
        st, it, rel = vfd.vfd_solve(ops[prec], Fb, U, rtol=1e-10, max_it=2)
        assert st == vfd.VFD_ENOCONV
        assert torch.isfinite(U).all().item()
        assert np.all(rel > 1e-10) and np.all(np.isfinite(rel))


def test_batch_noconv(setup):
    m, mesh, ops, F = setup
    m2 = synth.square_mesh_for_dofs(500, jitter=0.2, seed=5)
    mesh2 = vfd.vfd_mesh(2, m2.coords, m2.cells, m2.cell_is_interior, leaf_m=32, lam=0.75, rho_lambda=0.75)
    op2 = vfd.vfd_assemble(mesh2, synth.config2_s_field(), synth.const_field(0.0), 0.9, precision=vfd.VFD_FP32)
    b = vfd.vfd_batch_create([ops[vfd.VFD_FP32], op2])
    g = torch.Generator(device="cuda").manual_seed(4)
    Fs = [torch.randn(64, n, dtype=torch.float64, device="cuda", generator=g) for n in (mesh.n_dof, mesh2.n_dof)]
    Us = [torch.zeros_like(f) for f in Fs]
    st, it, rel = vfd.vfd_batch_solve(b, Fs, Us, rtol=1e-10, max_it=2)
    assert st == vfd.VFD_ENOCONV
    assert all(torch.isfinite(u).all().item() for u in Us)
    assert np.all(rel > 1e-10)


def test_bf16_column_path_equals_fp32(setup):
    m, mesh, ops, F = setup
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(3, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    Y32 = torch.empty_like(X)
    Y16 = torch.empty_like(X)
    vfd.vfd_apply(ops[vfd.VFD_FP32], X, Y32)
    vfd.vfd_apply(ops[vfd.VFD_BF16], X, Y16)
    torch.cuda.synchronize()
    assert torch.equal(Y32, Y16)
