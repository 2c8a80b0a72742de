"""Parity at the benchmark's full size: the 2D disk of 27,361 DoFs (34,027
vertices), the benchmark's fields and mesh options (leaf 64, Chebyshev p = 8,
lambda = 0.75, FP64), in the launch configuration bench.py times.

* sampled rows of A x against the oracle's exact rows (oracle.apply_rows,
  no approximation): exact-mode operator (every block near, direct density)
  to 1e-11; the benchmark's H^2 operator (rank 64) to the matvec tolerance
  1e-6 (its measured error is about 1e-7); the rank-16 operator (p = 4) to
  its interpolation error (about 3e-5);
* the FP64 CG solution's true residual, and the 64-RHS TF32 / BF16
  refinement's residuals through the FP64 operator;
* the adjoint gradient's log-kappa shift identity sum_k g_k = -Lam^T A U
  (holds at any size) on the benchmark H^2 operator with P1 fields, and the
  autograd gradient of a solution misfit against central differences along
  20 seeded directions (the differentiation workload at full size).
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402

NROWS = 48


@pytest.fixture(scope="module")
def disk():
    m, s, k, prm = synth.workload("disk33k")
    dof_o, N = oracle.dofs(m)
    return m, s, k, prm, dof_o, N


def _mesh(m, prm, lam, p=None):
    return vfd.vfd_mesh(m.d, m.coords, m.cells, m.cell_is_interior, leaf_m=prm["leaf"], cheb_p=p or prm["p"],
                        lam=lam, rho_lambda=lam, tail_mode=prm["tail"], tail_R=prm["R"])


def _sampled_rows(disk, lam, tol, p=None):
    m, s, k, prm, dof_o, N = disk
    mesh = _mesh(m, prm, lam, p)
    dof_g, n = vfd.vfd_mesh_dofs(mesh)
    assert n == N
    op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"])
    rng = np.random.default_rng(2024)
    xo = rng.standard_normal(N)
    sel = dof_g >= 0
    xg = np.zeros(n)
    xg[dof_g[sel]] = xo[dof_o[sel]]
    X = torch.tensor(xg, device="cuda")
    Y = torch.empty_like(X)
    vfd.vfd_apply(op, X, Y)
    torch.cuda.synchronize()
    yg = Y.cpu().numpy()
    verts = np.nonzero(sel)[0]
    pick = rng.choice(len(verts), NROWS, replace=False)
    rows_o = dof_o[verts[pick]]
    y_or = oracle.apply_rows(m, s, k, xo, rows_o, s_bar=prm["s_bar"], n_sing=3, tail=prm["tail"], R=prm["R"])
    y_gp = yg[dof_g[verts[pick]]]
    err = np.abs(y_gp - y_or).max() / np.abs(y_or).max()
    print(f"sampled rows, lambda {lam}: max error / max |y| = {err:.3e}")
    assert err < tol, err
    return err


def test_fullsize_exact_mode_sampled_rows(disk):
    _sampled_rows(disk, 0.0, 1e-11)


def test_fullsize_h2_sampled_rows(disk):
    # the benchmark operator: rank-64 Chebyshev interpolation of the far field
    # meets the matvec tolerance 1e-6 of the hot-path definition
    _sampled_rows(disk, 0.75, 1e-6)


def test_fullsize_rank16_sampled_rows(disk):
    # rank 16 (p = 4): the interpolation error is about 3e-5
    _sampled_rows(disk, 0.75, 1e-4, p=4)


def test_fullsize_solves(disk):
    m, s, k, prm, dof_o, N = disk
    mesh = _mesh(m, prm, 0.75)
    op = vfd.vfd_assemble(mesh, s, k, prm["s_bar"])
    F = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device="cuda"), F)
    U = torch.zeros_like(F)
    st, it, rel = vfd.vfd_solve(op, F, U, rtol=1e-10, max_it=100000)
    assert st == vfd.VFD_OK
    AU = torch.empty_like(U)
    vfd.vfd_apply(op, U, AU)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(F - AU) / torch.linalg.norm(F)).item() <= 1.01e-10
    g = torch.Generator(device="cuda").manual_seed(77)
    Fb = torch.randn(64, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    for prec in (vfd.VFD_FP32, vfd.VFD_BF16):
        opl = vfd.vfd_assemble(mesh, s, k, prm["s_bar"], precision=prec)
        Ub = torch.zeros_like(Fb)
        st, it, rel = vfd.vfd_solve(opl, Fb, Ub, rtol=1e-8, max_it=100000)
        assert st == vfd.VFD_OK
        AUb = torch.empty_like(Ub)
        vfd.vfd_apply(op, Ub, AUb)
        torch.cuda.synchronize()
        r = (torch.linalg.norm(Fb - AUb, dim=1) / torch.linalg.norm(Fb, dim=1)).max().item()
        assert r <= 1.01e-8, (prec, r)


def _fourier_values(f, x):
    """Vertex values of a synthetic Fourier field descriptor (input generation)."""
    v = np.full(len(x), float(f.c0))
    for row in np.asarray(f.fourier, dtype=float).reshape(-1, 5):
        v += row[3] * np.cos(math.pi * (x @ row[:2]) + row[4])
    return v


def _nodal(k, x):
    s_n = 0.25 + 0.5 * (0.5 + 0.5 * np.sin(2 * math.pi * x[:, 0]) * np.cos(2 * math.pi * x[:, 1]))
    return s_n, _fourier_values(k, x)


def test_fullsize_gradient_shift_identity(disk):
    """The benchmark's H^2 operator (rank 64) with P1 fields: the log-kappa
    shift identity sum_k g_k = -Lam^T A U, two columns."""
    m, s, k, prm, dof_o, N = disk
    s_n, lk_n = _nodal(k, m.coords)
    mesh = _mesh(m, prm, prm["lam"])
    op = vfd.vfd_assemble(mesh, synth.nodal_field(s_n), synth.nodal_field(lk_n), prm["s_bar"])
    g = torch.Generator(device="cuda").manual_seed(5)
    U = torch.randn(2, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    L = torch.randn(2, mesh.n_dof, dtype=torch.float64, device="cuda", generator=g)
    gs = torch.empty(m.n_vert, dtype=torch.float64, device="cuda")
    gk = torch.empty_like(gs)
    vfd.vfd_grad(op, U, L, gs, gk)
    AU = torch.empty_like(U)
    vfd.vfd_apply(op, U, AU)
    torch.cuda.synchronize()
    ref = -(L * AU).sum().item()
    assert abs(gk.sum().item() - ref) <= 1e-10 * abs(ref)


def test_fullsize_autograd_finite_differences(disk):
    """The differentiation workload at full size: nodal s and log kappa on the
    benchmark disk (H^2 operator, rank 64), loss = ||u - u_obs||^2 in the
    lumped mass norm with u_obs the solution for a seeded reference s field;
    the autograd gradient (adjoint solve + vfd_grad) against central
    differences (h = 1e-6) of the loss through the solve along 20 seeded
    directions in (s, log kappa) jointly."""
    from paper_2302_02863_gb300 import inverse
    from paper_2302_02863_gb300.autograd import solve as vsolve

    m, s, k, prm, dof_o, N = disk
    x = m.coords
    s_n, lk_n = _nodal(k, x)
    s_ref = np.clip(s_n + 0.05 * np.sin(3.0 * x[:, 0] + 1.0) * np.cos(2.0 * x[:, 1]), 0.1, 0.85)
    mesh = _mesh(m, prm, prm["lam"])
    dev = "cuda"
    F = torch.zeros(mesh.n_dof, dtype=torch.float64, device=dev)
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device=dev), F)
    m_l = inverse.lumped_mass(mesh, m.n_vert, dev)
    lk_t = torch.tensor(lk_n, device=dev)
    rtol = 1e-12
    with torch.no_grad():
        u_obs = vsolve(torch.tensor(s_ref, device=dev), lk_t, F, mesh, prm["s_bar"], rtol)

    def J(sv, lv):
        e = vsolve(sv, lv, F, mesh, prm["s_bar"], rtol) - u_obs
        return (m_l * e * e).sum()

    s_t = torch.tensor(s_n, device=dev, requires_grad=True)
    l_t = torch.tensor(lk_n, device=dev, requires_grad=True)
    J(s_t, l_t).backward()
    rng = np.random.default_rng(4)
    h = 1e-6
    worst = 0.0
    with torch.no_grad():
        for _ in range(20):
            vs = torch.tensor(rng.standard_normal(m.n_vert), device=dev)
            vl = torch.tensor(rng.standard_normal(m.n_vert), device=dev)
            fd = (J(s_t + h * vs, l_t + h * vl) - J(s_t - h * vs, l_t - h * vl)).item() / (2 * h)
            ad = ((s_t.grad * vs).sum() + (l_t.grad * vl).sum()).item()
            worst = max(worst, abs(ad - fd) / abs(fd))
    print(f"full-size autograd vs FD (20 directions, h = 1e-6): max rel gap {worst:.3e}")
    assert worst < 1e-6, worst   # measured 1.4e-7


def test_fullsize_h2_all_rows_vs_exact_mode(disk):
    """Every row of the benchmark operator against the exact-mode operator of the
    same disk (every block near, direct density: the quadrature matrix itself,
    equal to the oracle's rows to 1e-11 above): relative 2-norm error of A x
    below the matvec tolerance 1e-6 (measured about 1.5e-7, dominated by the
    density sweep), and above it for rank 16 (about 3e-5)."""
    m, s, k, prm, dof_o, N = disk
    mx = _mesh(m, prm, 0.0)
    opx = vfd.vfd_assemble(mx, s, k, prm["s_bar"])
    g = torch.Generator(device="cuda").manual_seed(8)
    X = torch.randn(mx.n_dof, dtype=torch.float64, device="cuda", generator=g)
    Yx = torch.empty_like(X)
    vfd.vfd_apply(opx, X, Yx)
    errs = {}
    for p in (prm["p"], 4):
        mh = _mesh(m, prm, 0.75, p)
        op = vfd.vfd_assemble(mh, s, k, prm["s_bar"])
        Y = torch.empty_like(X)
        vfd.vfd_apply(op, X, Y)
        torch.cuda.synchronize()
        errs[p] = (torch.linalg.norm(Y - Yx) / torch.linalg.norm(Yx)).item()
    print(f"all rows vs exact mode: {errs}")
    assert errs[prm["p"]] < 1e-6
    assert errs[4] > 1e-6
