"""vfd_apply_noalloc: the apply whose far-field scratch is a fixed static device
array, so that the call allocates nothing.

Checked against vfd_apply (same operator, same kernels) on two calls in a
row, for FP64, FP32 and BF16 operators (the last two apply K in FP32 column
by column) and one and several columns; with a leading dimension larger than
the number of DoFs; after a call that left the scratch holding values of
another layout (no entry of the scratch needs an initial value); and that the
sizes the static scratch cannot hold, and host pointers, are rejected before
anything runs.  The file name makes pytest collect it last.
"""
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


@pytest.fixture(scope="module")
def mesh():
    m = synth.disk_mesh(14, R=1.1, jitter=0.2, seed=9)
    h = vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=32, lam=0.75, rho_lambda=0.75)
    assert h.info["far_blocks"] > 0 and h.info["near_blocks"] > 0
    return h


@pytest.fixture(scope="module")
def ops(mesh):
    s = synth.config2_s_field()
    k = synth.random_fourier_field(31, 0.5)
    return {p: vfd.vfd_assemble(mesh, s, k, 0.9, precision=p) for p in (vfd.VFD_FP64, vfd.VFD_FP32, vfd.VFD_BF16)}


def _rel(Y, Yref):
    return (torch.linalg.norm(Y - Yref, dim=-1) / torch.linalg.norm(Yref, dim=-1)).max().item()


@pytest.mark.parametrize("prec", [vfd.VFD_FP64, vfd.VFD_FP32, vfd.VFD_BF16])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_matches_apply_twice(mesh, ops, prec, nrhs):
    op = ops[prec]
    g = torch.Generator(device="cpu").manual_seed(100 + nrhs)
    X = torch.randn(nrhs, mesh.n_dof, dtype=torch.float64, generator=g).cuda()
    Yref = torch.empty_like(X)
    vfd.vfd_apply(op, X, Yref)
    torch.cuda.synchronize()
    # same kernels in the same order on one stream: equal up to rounding noise
    tol = 1e-12
    for _ in range(2):
        Y = torch.full_like(X, float("nan"))
        vfd.vfd_apply_noalloc(op, X, Y)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(Y - Yref, dim=1) / torch.linalg.norm(Yref, dim=1)).max().item()
        assert err <= tol, err


def test_noalloc_leading_dimension(mesh, ops):
    # columns of length n_dof + 7: the library reads and writes the first n_dof
    # entries of each column only
    n, ld, nrhs = mesh.n_dof, mesh.n_dof + 7, 3
    g = torch.Generator(device="cpu").manual_seed(7)
    X = torch.randn(nrhs, ld, dtype=torch.float64, generator=g).cuda()
    for prec in (vfd.VFD_FP64, vfd.VFD_FP32):
        Yref = torch.full_like(X, 5.0)
        vfd.vfd_apply(ops[prec], X, Yref)
        Y = torch.full_like(X, 5.0)
        vfd.vfd_apply_noalloc(ops[prec], X, Y)
        torch.cuda.synchronize()
        assert _rel(Y[:, :n], Yref[:, :n]) <= 1e-12
        assert torch.all(Y[:, n:] == 5.0).item()   # the 7 padding entries untouched


def test_noalloc_stale_scratch(mesh, ops):
    # a wide FP32 call fills the scratch with FP32 partial sums in its own
    # layout; the next FP64 single-column call must not depend on them
    n = mesh.n_dof
    g = torch.Generator(device="cpu").manual_seed(8)
    Xw = torch.randn(6, n, dtype=torch.float64, generator=g).cuda()
    x1 = torch.randn(n, dtype=torch.float64, generator=g).cuda()
    Yw_ref = torch.empty_like(Xw)
    y1_ref = torch.empty_like(x1)
    vfd.vfd_apply(ops[vfd.VFD_FP32], Xw, Yw_ref)
    vfd.vfd_apply(ops[vfd.VFD_FP64], x1, y1_ref)
    for _ in range(2):
        Yw = torch.empty_like(Xw)
        y1 = torch.empty_like(x1)
        vfd.vfd_apply_noalloc(ops[vfd.VFD_FP32], Xw, Yw)
        vfd.vfd_apply_noalloc(ops[vfd.VFD_FP64], x1, y1)
        torch.cuda.synchronize()
        assert _rel(Yw, Yw_ref) <= 1e-12
        assert _rel(y1, y1_ref) <= 1e-12


def test_noalloc_rejects_oversize(mesh, ops):
    info = mesh.info
    # the node sums alone (2 x nodes x rank doubles per column) exceed the scratch
    nrhs = math.ceil(vfd.VFD_APPLY_NOALLOC_SCRATCH_BYTES / (2 * info["nodes"] * info["rank"] * 8)) + 1
    X = torch.ones(nrhs, mesh.n_dof, dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(vfd.VfdError) as e:
        vfd.vfd_apply_noalloc(ops[vfd.VFD_FP64], X, Y)
    assert e.value.status == vfd.VFD_EINVAL
    assert str(vfd.VFD_APPLY_NOALLOC_SCRATCH_BYTES) in str(e.value)
    torch.cuda.synchronize()
    assert torch.count_nonzero(Y).item() == 0   # nothing ran


def test_noalloc_rejects_host_pointers(mesh, ops):
    X = np.ones(mesh.n_dof)
    Y = np.zeros(mesh.n_dof)
    with pytest.raises(vfd.VfdError) as e:
        vfd.vfd_apply_noalloc(ops[vfd.VFD_FP64], X, Y)
    assert e.value.status == vfd.VFD_EINVAL
    assert not Y.any()
