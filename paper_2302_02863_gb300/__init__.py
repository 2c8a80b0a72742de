"""GB300 (sm_103a) implementation of the linear-complexity finite element
operator for variable-order fractional diffusion (Lei, Turkiyyah & Knio,
arXiv 2302.02863): A = B + K_H2 + M_w assembled and applied on the device,
with a device-resident CG / iterative-refinement solver.

The compute path is the CUDA library libvfd.so (C ABI in include/vfd.h);
`vfd` is its ctypes binding.
"""
from . import vfd  # noqa: F401

__all__ = ["vfd"]
