"""Adjoint gradient on the GPU (vfd_grad) and the autograd wrapper.

* vfd_grad against the oracle's gradient (the derivative of the dense
  route-2 matrix, pinned by finite differences in test_oracle_grad.py) for
  the same U and Lam, element by element over all vertices: 2D and 1D, one
  and ten columns (ten: two passes of the separated-pair kernel);
* the dense-oracle comparison on a disk of 1,951 vertices;
* the autograd Function against central finite differences of the GPU solve.
Tolerances: the GPU sums the same terms in another order with a table-driven
log/exp (relative error ~1e-16 per evaluation), so 1e-10 of max|g|.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402
from paper_2302_02863_gb300.autograd import solve as vsolve  # noqa: E402

SBAR = 0.9


def _fields(m, seed):
    rng = np.random.default_rng(seed)
    x = m.coords
    s = 0.45 + 0.15 * np.sin(2.0 * x[:, 0]) + 0.05 * rng.standard_normal(m.n_vert)
    lk = 0.3 * np.cos(1.5 * x[:, -1]) + 0.1 * rng.standard_normal(m.n_vert)
    return np.clip(s, 0.15, 0.8), lk


def _exact_mesh(m, leaf=32):
    return vfd.vfd_mesh(m.d, m.coords, m.cells, m.cell_is_interior, leaf_m=leaf, lam=0.0, rho_lambda=0.0)


def _compare(m, nrhs, seed, U_from_solve=False):
    s, lk = _fields(m, seed)
    mesh = _exact_mesh(m)
    op = vfd.vfd_assemble(mesh, synth.nodal_field(s), synth.nodal_field(lk), SBAR)
    dof_g, n = vfd.vfd_mesh_dofs(mesh)
    dof_o, N = oracle.dofs(m)
    assert n == N
    sel = dof_g >= 0
    rng = np.random.default_rng(seed + 1)
    Uo = rng.standard_normal((nrhs, N))
    Lo = rng.standard_normal((nrhs, N))
    if U_from_solve:
        F = torch.zeros(n, dtype=torch.float64, device="cuda")
        vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device="cuda"), F)
        U1 = torch.zeros_like(F)
        vfd.vfd_solve(op, F, U1, rtol=1e-12, max_it=100000, raise_on_noconv=True)
        Uo[0, dof_o[sel]] = U1.cpu().numpy()[dof_g[sel]]
    Ug = np.zeros((nrhs, n))
    Lg = np.zeros((nrhs, n))
    Ug[:, dof_g[sel]] = Uo[:, dof_o[sel]]
    Lg[:, dof_g[sel]] = Lo[:, dof_o[sel]]
    U = torch.tensor(Ug, device="cuda")
    L = torch.tensor(Lg, device="cuda")
    gs = torch.empty(m.n_vert, dtype=torch.float64, device="cuda")
    gk = torch.empty_like(gs)
    vfd.vfd_grad(op, U[0] if nrhs == 1 else U, L[0] if nrhs == 1 else L, gs, gk)
    gs_o, gk_o = oracle.grad(m, s, lk, Uo, Lo, s_bar=SBAR, n_sing=3)
    for g, go in ((gs.cpu().numpy(), gs_o), (gk.cpu().numpy(), gk_o)):
        err = np.abs(g - go).max() / np.abs(go).max()
        assert err < 1e-10, err


@pytest.mark.parametrize("nrhs", [1, 10])
def test_grad_matches_oracle_2d(nrhs):
    _compare(synth.disk_mesh(6, R=1.1, jitter=0.2, seed=8), nrhs, seed=40 + nrhs)


def test_grad_matches_oracle_1d():
    _compare(synth.interval_mesh(40, R=1.2), 3, seed=50)


def test_grad_dense_oracle_2k_vertices():
    # the 1,951-vertex disk; U from the GPU solve with f = 1, Lam random
    _compare(synth.disk_mesh(23, R=1.1, jitter=0.2, seed=2023), 1, seed=60, U_from_solve=True)


def test_autograd_matches_finite_differences():
    m = synth.disk_mesh(4, R=1.1, jitter=0.2, seed=9)
    s0, lk0 = _fields(m, 70)
    mesh = _exact_mesh(m, leaf=16)
    F = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
    vfd.vfd_load(mesh, torch.ones(m.n_vert, dtype=torch.float64, device="cuda"), F)
    g = torch.Generator(device="cpu").manual_seed(3)
    U_obs = torch.randn(mesh.n_dof, dtype=torch.float64, generator=g).cuda() * 0.1

    def J(s, lk):
        U = vsolve(s, lk, F, mesh, SBAR, 1e-12)
        return ((U - U_obs) ** 2).sum()

    s = torch.tensor(s0, device="cuda", requires_grad=True)
    lk = torch.tensor(lk0, device="cuda", requires_grad=True)
    J(s, lk).backward()
    h = 1e-5
    rng = np.random.default_rng(71)
    for which in ("s", "lk"):
        for _ in range(3):
            v = torch.tensor(rng.standard_normal(m.n_vert), device="cuda")
            with torch.no_grad():
                if which == "s":
                    fd = (J(s + h * v, lk) - J(s - h * v, lk)) / (2 * h)
                    ad = (s.grad * v).sum()
                else:
                    fd = (J(s, lk + h * v) - J(s, lk - h * v)) / (2 * h)
                    ad = (lk.grad * v).sum()
            assert abs(ad.item() - fd.item()) <= 1e-5 * abs(fd.item()), (which, ad.item(), fd.item())


def test_grad_rejects_analytic_fields():
    m = synth.disk_mesh(3, R=1.1, jitter=0.2, seed=5)
    mesh = _exact_mesh(m)
    op = vfd.vfd_assemble(mesh, synth.config2_s_field(), synth.const_field(0.0), SBAR)
    U = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
    g = torch.empty(m.n_vert, dtype=torch.float64, device="cuda")
    with pytest.raises(vfd.VfdError) as e:
        vfd.vfd_grad(op, U, U, g, g.clone())
    assert e.value.status == vfd.VFD_EUNSUPPORTED
