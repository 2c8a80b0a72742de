"""Batches of operators (several meshes, one launch per stage, one batched
refinement solve).

* vfd_batch_apply on three meshes (a disk and a square with far blocks, a
  small disk without) against vfd_apply of each operator alone (the same
  kernels per mesh: equal to rounding);
* vfd_batch_solve to 1e-8: the FP64 residual of every column of every mesh
  through the FP64 operators, and the exact-mode mesh against the oracle's
  Cholesky solution.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


def _setup(prec):
    cases = [
        (synth.disk_mesh(12, R=1.1, jitter=0.2, seed=31), 0.75, 1),
        (synth.square_mesh(32, jitter=0.2, seed=32), 0.75, 2),
        (synth.disk_mesh(6, R=1.1, jitter=0.2, seed=33), 0.0, 3),
    ]
    out = []
    for m, lam, seed in cases:
        mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=lam, rho_lambda=lam)
        s = synth.sigmoid_field(synth.random_fourier_field(100 + seed, 1.0), 0.1, 0.9)
        k = synth.random_fourier_field(200 + seed, 0.5)
        op64 = vfd.vfd_assemble(mesh, s, k, 0.9)
        opl = vfd.vfd_assemble(mesh, s, k, 0.9, precision=prec)
        out.append((m, mesh, s, k, op64, opl, lam))
    assert out[0][1].info["far_blocks"] > 0 and out[1][1].info["far_blocks"] > 0
    assert out[2][1].info["far_blocks"] == 0
    return out


@pytest.mark.parametrize("prec", [vfd.VFD_FP32, vfd.VFD_BF16])
def test_batch_apply_matches_single(prec):
    cases = _setup(prec)
    batch = vfd.vfd_batch_create([c[5] for c in cases])
    g = torch.Generator(device="cuda").manual_seed(5)
    Xs = [torch.randn(64, c[1].n_dof, dtype=torch.float64, device="cuda", generator=g) for c in cases]
    Ys = [torch.empty_like(x) for x in Xs]
    vfd.vfd_batch_apply(batch, Xs, Ys)
    chosen, us = vfd.vfd_batch_tuning(batch)
    assert chosen[0] > 0 and chosen[2] >= 1 and max(us) > 0   # a near-panel configuration was timed and picked
    for c, x, y in zip(cases, Xs, Ys):
        ref = torch.empty_like(x)
        vfd.vfd_apply(c[5], x, ref)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-6, err


@pytest.mark.parametrize("prec", [vfd.VFD_FP32, vfd.VFD_BF16])
def test_batch_solve(prec):
    cases = _setup(prec)
    batch = vfd.vfd_batch_create([c[5] for c in cases])
    g = torch.Generator(device="cuda").manual_seed(6)
    Fs = [torch.randn(64, c[1].n_dof, dtype=torch.float64, device="cuda", generator=g) for c in cases]
    Us = [torch.zeros_like(f) for f in Fs]
    st, it, rel = vfd.vfd_batch_solve(batch, Fs, Us, rtol=1e-8, max_it=50000)
    assert st == vfd.VFD_OK and rel.shape == (3, 64) and np.all(rel <= 1e-8), (st, rel.max())
    for c, F, U in zip(cases, Fs, Us):
        AU = torch.empty_like(U)
        vfd.vfd_apply(c[4], U, AU)
        torch.cuda.synchronize()
        r = (torch.linalg.norm(F - AU, dim=1) / torch.linalg.norm(F, dim=1)).max().item()
        assert r <= 1.5e-8, r
    # the exact-mode mesh against the oracle's dense Cholesky solution
    m, mesh, s, k = cases[2][:4]
    ref = oracle.assemble(m, s, k, s_bar=0.9, n_sing=3)
    dof, n = vfd.vfd_mesh_dofs(mesh)
    sel = dof >= 0
    Fo = np.zeros((64, n))
    Fo[:, ref.dof[sel]] = Fs[2].cpu().numpy()[:, dof[sel]]
    L = np.linalg.cholesky(ref.A)
    Uo = np.linalg.solve(L.T, np.linalg.solve(L, Fo.T)).T
    Ug = Us[2].cpu().numpy()[:, dof[sel]]
    err = np.linalg.norm(Ug - Uo[:, ref.dof[sel]], axis=1) / np.linalg.norm(Uo, axis=1)
    assert err.max() < 1e-6, err.max()


def test_batch_rejects_mixed_precision():
    cases = _setup(vfd.VFD_FP32)
    opb = vfd.vfd_assemble(cases[2][1], cases[2][2], cases[2][3], 0.9, precision=vfd.VFD_BF16)
    with pytest.raises(vfd.VfdError):
        vfd.vfd_batch_create([cases[0][5], opb])
    with pytest.raises(vfd.VfdError):
        vfd.vfd_batch_create([cases[0][4]])   # FP64 operator


def test_preconditioned_low_precision_on_hard_mesh():
    """Mesh 13 of the 24-mesh workload (a 21k-DoF disk, s in [0.1, 0.9]):
    with x rounded once to BF16 before the near-panel product, the
    preconditioned inner iteration took 1253 BF16 steps (TF32: 80-152); with x
    carried as hi + lo terms it takes about 40 in both precisions."""
    i = 13
    n = int(round(2000 * 65.0 ** (i / 23)))
    m = synth.disk_mesh_for_dofs(n, R=1.1, jitter=0.2, seed=3000 + i)
    s = synth.sigmoid_field(synth.random_fourier_field(3000 + i + 100, 1.0), 0.1, 0.9)
    k = synth.random_fourier_field(3000 + i + 200, 0.5)
    mesh = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=64, cheb_p=4, lam=0.75, rho_lambda=0.75)
    op64 = vfd.vfd_assemble(mesh, s, k, 0.9)
    g = torch.Generator(device="cuda").manual_seed(4013)
    F = torch.randn(64, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    for prec in (vfd.VFD_BF16, vfd.VFD_FP32):
        op = vfd.vfd_assemble(mesh, s, k, 0.9, precision=prec)
        vfd.vfd_precondition(op)
        batch = vfd.vfd_batch_create([op])
        for bad in (0.0, 1.0, -0.5, float("nan")):
            with pytest.raises(vfd.VfdError):
                vfd.vfd_batch_set_update_drop(batch, bad)
        vfd.vfd_batch_set_update_drop(batch, 0.03)
        U = torch.zeros_like(F)
        st, it, rel = vfd.vfd_batch_solve(batch, [F], [U], rtol=1e-8, max_it=2000)
        assert st == vfd.VFD_OK and rel.max() <= 1e-8
        assert it.max() <= 120, (prec, it.max())
        R = F - vfd.vfd_apply(op64, U, torch.empty_like(U))
        assert (torch.linalg.norm(R, dim=1) / torch.linalg.norm(F, dim=1)).max().item() <= 1e-8
