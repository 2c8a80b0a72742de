"""The library's table-driven FP64 log / exp (used for every kernel
evaluation) against numpy's (correctly rounded to within an ulp) on the
ranges the kernel evaluations reach, through the C ABI."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_02863_gb300 import vfd  # noqa: E402


@pytest.fixture(scope="module")
def mesh():
    m = synth.disk_mesh(3, R=1.3, jitter=0.0)
    return vfd.vfd_mesh(2, m.coords, m.cells, m.cell_is_interior, leaf_m=8)


def test_log_accuracy(mesh):
    rng = np.random.default_rng(0)
    x = np.concatenate([np.exp(rng.uniform(-40, 10, 200000)), rng.uniform(0.5, 2.0, 100000),
                        np.array([1.0, 2.0, 0.5, 1e-300, 1e300, 1.0 + 2e-16, 1.0 - 1e-16])])
    X = torch.tensor(x, device="cuda")
    Y = torch.empty_like(X)
    vfd.vfd_selftest_math(mesh, 0, X, Y)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    ref = np.log(x)
    err = np.abs(y - ref)
    # absolute error a few ulp of max(|log x|, 1) (what enters exp(a - b log r^2))
    assert np.max(err / np.maximum(np.abs(ref), 1.0)) < 8e-16


def test_exp_accuracy(mesh):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-690, 690, 200000), rng.uniform(-5, 5, 200000),
                        np.array([0.0, 1.0, -1.0, 1e-12, -1e-12, 700.0, -700.0])])
    X = torch.tensor(x, device="cuda")
    Y = torch.empty_like(X)
    vfd.vfd_selftest_math(mesh, 1, X, Y)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    ref = np.exp(x)
    rel = np.abs(y - ref) / ref
    assert np.max(rel) < 4e-16


@pytest.mark.parametrize("which,fn", [(2, np.cos), (3, np.sin)])
def test_trig_pi_accuracy(mesh, which, fn):
    """The table-driven cos / sin of pi x used for the Fourier fields, against an
    extended-precision reference (long double, pi from 4 atan 1)."""
    rng = np.random.default_rng(2 + which)
    x = np.concatenate([rng.uniform(-2.5, 2.5, 200000), rng.uniform(-40, 40, 20000),
                        np.array([0.0, 0.5, 1.0, -1.0, 1.0 / 128, -1.0 / 128, 0.25, 2.0])])
    X = torch.tensor(x, device="cuda")
    Y = torch.empty_like(X)
    vfd.vfd_selftest_math(mesh, which, X, Y)
    torch.cuda.synchronize()
    y = Y.cpu().numpy()
    pi = 4 * np.arctan(np.longdouble(1))
    ref = fn(pi * x.astype(np.longdouble)).astype(np.float64)
    assert np.max(np.abs(y - ref)) < 4e-16
