"""vfd_apply_noalloc: the apply whose far-field scratch is a fixed static device
array, so that the call allocates nothing.

Checked against vfd_apply (same operator, same kernels) on two calls in a
row, for FP64 and FP32 operators and one and several columns; and that the
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
    return {p: vfd.vfd_assemble(mesh, s, k, 0.9, precision=p) for p in (vfd.VFD_FP64, vfd.VFD_FP32)}


@pytest.mark.parametrize("prec", [vfd.VFD_FP64, vfd.VFD_FP32])
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
