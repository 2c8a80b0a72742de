"""The C-ABI library builds, loads without a GPU and exports every function
declared in include/vfd.h; without a CUDA device its compute entry points
fail with VFD_ECUDA instead of falling back to the CPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "vfd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vfd_[a-z_]+)\s*\(", txt)))


def test_exports_match_header():
    import __graft_entry__ as g
    g.build()
    from paper_2302_02863_gb300 import vfd
    L = vfd.load()
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), f"libvfd.so does not export {n}"
    assert set(names) == set(vfd.EXPORTS)


def test_no_cpu_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2302_02863_gb300 import vfd
    X = np.array([[0.0], [0.5], [1.0]])
    T = np.array([[0, 1], [1, 2]], dtype=np.int32)
    with pytest.raises(vfd.VfdError) as e:
        vfd.vfd_mesh(1, X, T, np.array([1, 1], dtype=np.uint8))
    assert e.value.status == vfd.VFD_ECUDA


def test_default_options():
    from paper_2302_02863_gb300 import vfd
    o = vfd.vfd_default_mesh_opts()
    assert (o.leaf_m, o.cheb_p, o.n_sing) == (64, 4, 3)
    assert abs(o.lam - 0.75) < 1e-15 and abs(o.tail_R - 1.1) < 1e-15
