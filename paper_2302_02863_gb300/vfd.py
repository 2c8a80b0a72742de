"""Thin ctypes binding of the vfd C ABI (include/vfd.h).

Argument marshalling only: every step of the operator (assembly, apply,
solve) runs in the CUDA kernels of libvfd.so.  Arrays may be torch CUDA
tensors (device pointers, the caller's stream) or numpy / CPU arrays (host
pointers; the library stages them).  Multi-RHS blocks are passed as arrays of
shape (nrhs, n_dof): row r is right-hand side r, i.e. column-major with
ld = n_dof in the C ABI's terms.

There is no CPU fallback: if libvfd.so is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvfd.so")

VFD_OK, VFD_EINVAL, VFD_ENOMEM, VFD_ECUDA, VFD_ENOCONV, VFD_ETIMEOUT, VFD_EUNSUPPORTED = range(7)
VFD_FP64, VFD_FP32, VFD_BF16 = 0, 1, 2
VFD_PART_B, VFD_PART_M, VFD_PART_KNEAR, VFD_PART_KFAR, VFD_PART_ALL = 1, 2, 4, 8, 15
VFD_PREC_NONE, VFD_PREC_TWO_LEVEL, VFD_PREC_BLOCK_JACOBI = 0, 1, 2
VFD_ASSEMBLE_UNCHECKED = 1
VFD_ASSEMBLE_TIMED = 2
VFD_APPLY_NOALLOC_SCRATCH_BYTES = 8388608   # static scratch of vfd_apply_noalloc, per device
TIMING_KEYS = ["fields", "coupling", "near", "density", "singular", "gather", "total"]
VFD_FIELD_ANALYTIC, VFD_FIELD_NODAL = 0, 1
INFO_KEYS = ["n_dof", "n_vert", "n_cell", "touching_pairs", "nnz", "levels", "nodes", "rank",
             "far_blocks", "near_blocks", "near_entries", "n_q", "n_qint", "rho_far_blocks",
             "rho_near_pairs", "near_storage", "near_point_pairs", "sing_points", "inner_rank"]

EXPORTS = ["vfd_default_mesh_opts", "vfd_mesh", "vfd_mesh_dofs", "vfd_mesh_info", "vfd_assemble",
           "vfd_apply", "vfd_apply_parts", "vfd_apply_noalloc", "vfd_solve", "vfd_precondition", "vfd_grad", "vfd_load",
           "vfd_op_rho", "vfd_op_timings", "vfd_op_far_ranks",
           "vfd_selftest_math", "vfd_batch_create", "vfd_batch_apply", "vfd_batch_solve", "vfd_batch_tuning",
           "vfd_batch_set_config", "vfd_batch_set_wait_limit", "vfd_batch_set_update_drop", "vfd_batch_free",
           "vfd_free_op", "vfd_free_mesh", "vfd_last_error"]


class VfdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"vfd status {status}: {msg}")
        self.status = status


class MeshOpts(C.Structure):
    _fields_ = [("leaf_m", C.c_int), ("cheb_p", C.c_int), ("lam", C.c_double), ("n_sing", C.c_int),
                ("tail_mode", C.c_int), ("tail_R", C.c_double), ("rho_leaf_m", C.c_int),
                ("rho_lambda", C.c_double), ("inner_p", C.c_int), ("recompress_tol", C.c_double)]


class FieldStruct(C.Structure):
    _fields_ = [("kind", C.c_int), ("c0", C.c_double), ("n_fourier", C.c_int),
                ("fourier", C.POINTER(C.c_double)), ("n_gauss", C.c_int), ("gauss", C.POINTER(C.c_double)),
                ("n_tbump", C.c_int), ("tbump", C.POINTER(C.c_double)), ("squash", C.c_int),
                ("lo", C.c_double), ("hi", C.c_double), ("nodal", C.POINTER(C.c_double))]


_lib = None


def load():
    """Load libvfd.so (built by __graft_entry__.build() / _build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.vfd_default_mesh_opts.argtypes = [C.POINTER(MeshOpts)]
    L.vfd_default_mesh_opts.restype = None
    L.vfd_mesh.argtypes = [C.c_int, C.c_int64, dp, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_uint8),
                           C.POINTER(MeshOpts), C.POINTER(vp)]
    L.vfd_mesh_dofs.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]
    L.vfd_mesh_info.argtypes = [vp, C.POINTER(C.c_int64), C.c_int]
    L.vfd_assemble.argtypes = [vp, C.POINTER(FieldStruct), C.POINTER(FieldStruct), C.c_double, C.c_int,
                               C.c_int, vp, C.POINTER(vp)]
    L.vfd_apply.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, vp]
    L.vfd_apply_parts.argtypes = [vp, C.c_int, vp, vp, C.c_int64, C.c_int64, vp]
    L.vfd_apply_noalloc.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, vp]
    L.vfd_grad.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, vp, vp, vp]
    L.vfd_solve.argtypes = [vp, vp, vp, C.c_int64, C.c_int64, C.c_double, C.c_int, C.POINTER(C.c_int),
                            dp, vp]
    L.vfd_load.argtypes = [vp, vp, vp, vp]
    L.vfd_precondition.argtypes = [vp, C.c_int, vp]
    L.vfd_op_rho.argtypes = [vp, vp, vp]
    L.vfd_op_timings.argtypes = [vp, dp, C.c_int]
    L.vfd_op_far_ranks.argtypes = [vp, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    L.vfd_selftest_math.argtypes = [vp, C.c_int, C.c_int64, vp, vp, vp]
    L.vfd_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp)]
    L.vfd_batch_apply.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int64), C.c_int64, vp]
    L.vfd_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int64), C.c_int64, C.c_double,
                                  C.c_int, C.POINTER(C.c_int), dp, vp]
    L.vfd_batch_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]
    L.vfd_batch_set_config.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
    L.vfd_batch_set_wait_limit.argtypes = [vp, C.c_double]
    L.vfd_batch_set_update_drop.argtypes = [vp, C.c_double]
    L.vfd_batch_free.argtypes = [vp]
    L.vfd_batch_free.restype = None
    L.vfd_free_op.argtypes = [vp]
    L.vfd_free_op.restype = None
    L.vfd_free_mesh.argtypes = [vp]
    L.vfd_free_mesh.restype = None
    L.vfd_last_error.restype = C.c_char_p
    for f in ["vfd_mesh", "vfd_mesh_dofs", "vfd_mesh_info", "vfd_assemble", "vfd_apply", "vfd_apply_parts",
              "vfd_apply_noalloc", "vfd_grad", "vfd_batch_create", "vfd_batch_apply", "vfd_batch_solve",
              "vfd_batch_tuning", "vfd_batch_set_config", "vfd_batch_set_wait_limit", "vfd_batch_set_update_drop",
              "vfd_solve", "vfd_precondition", "vfd_load", "vfd_op_rho", "vfd_op_timings", "vfd_op_far_ranks",
              "vfd_selftest_math"]:
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(st):
    if st != VFD_OK:
        raise VfdError(st, load().vfd_last_error().decode())
    return st


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (no copies here)."""
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch tensor or a numpy array")


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


def _nrhs_ld(a, n):
    if a.ndim == 1:
        return 1, n
    return a.shape[0], a.shape[1]


class Mesh:
    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().vfd_free_mesh(self.handle)
            except Exception:
                pass
            self.handle = None


class Op:
    def __init__(self, handle, mesh, keep):
        self.handle = handle
        self.mesh = mesh
        self._keep = keep

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().vfd_free_op(self.handle)
            except Exception:
                pass
            self.handle = None


def vfd_default_mesh_opts():
    o = MeshOpts()
    load().vfd_default_mesh_opts(C.byref(o))
    return o


def vfd_mesh(d, coords, cells, cell_is_interior, opts=None, **kw):
    """Build a mesh handle (host arrays).  kw overrides fields of the default
    options (leaf_m, cheb_p, lam, n_sing, tail_mode, tail_R, rho_leaf_m, rho_lambda, inner_p,
    recompress_tol)."""
    L = load()
    o = vfd_default_mesh_opts() if opts is None else opts
    for k, v in kw.items():
        setattr(o, k, v)
    X = np.ascontiguousarray(coords, dtype=np.float64)
    T = np.ascontiguousarray(cells, dtype=np.int32)
    I = np.ascontiguousarray(cell_is_interior, dtype=np.uint8)
    h = C.c_void_p()
    _check(L.vfd_mesh(int(d), X.shape[0], X.ctypes.data_as(C.POINTER(C.c_double)), T.shape[0],
                      T.ctypes.data_as(C.POINTER(C.c_int32)), I.ctypes.data_as(C.POINTER(C.c_uint8)),
                      C.byref(o), C.byref(h)))
    m = Mesh(h, None)
    m.n_vert = X.shape[0]
    m.d = d
    m.info = vfd_mesh_info(m)
    m.n_dof = m.info["n_dof"]
    return m


def vfd_mesh_dofs(mesh):
    dof = np.zeros(mesh.n_vert, dtype=np.int32)
    n = C.c_int64()
    _check(load().vfd_mesh_dofs(mesh.handle, dof.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(n)))
    return dof, int(n.value)


def vfd_mesh_info(mesh):
    a = np.zeros(len(INFO_KEYS), dtype=np.int64)
    _check(load().vfd_mesh_info(mesh.handle, a.ctypes.data_as(C.POINTER(C.c_int64)), len(a)))
    return dict(zip(INFO_KEYS, (int(x) for x in a)))


def _field(f, keep):
    fs = FieldStruct()
    nodal = getattr(f, "nodal", None)
    if nodal is not None:
        fs.kind = VFD_FIELD_NODAL
        if isinstance(nodal, np.ndarray):
            nodal = np.ascontiguousarray(nodal, dtype=np.float64)
        keep.append(nodal)
        fs.nodal = C.cast(_ptr(nodal), C.POINTER(C.c_double))
        return fs
    fs.kind = VFD_FIELD_ANALYTIC
    fs.c0 = float(f.c0)
    for name in ("fourier", "gauss", "tbump"):
        rows = np.ascontiguousarray(np.asarray(getattr(f, name, np.zeros((0, 5))), dtype=np.float64).reshape(-1, 5))
        keep.append(rows)
        setattr(fs, "n_" + name, rows.shape[0])
        setattr(fs, name, rows.ctypes.data_as(C.POINTER(C.c_double)))
    fs.squash = int(getattr(f, "squash", 0))
    fs.lo = float(getattr(f, "lo", 0.0))
    fs.hi = float(getattr(f, "hi", 1.0))
    return fs


def vfd_assemble(mesh, s, log_kappa, s_bar, precision=VFD_FP64, flags=0, stream=None):
    keep = []
    fs = _field(s, keep)
    fk = _field(log_kappa, keep)
    h = C.c_void_p()
    _check(load().vfd_assemble(mesh.handle, C.byref(fs), C.byref(fk), float(s_bar), int(precision), int(flags),
                               _stream(stream), C.byref(h)))
    return Op(h, mesh, None)


def vfd_apply(op, X, Y, stream=None):
    nrhs, ld = _nrhs_ld(X, op.mesh.n_dof)
    _check(load().vfd_apply(op.handle, _ptr(X), _ptr(Y), nrhs, ld, _stream(stream)))
    return Y


def vfd_apply_parts(op, parts, X, Y, stream=None):
    nrhs, ld = _nrhs_ld(X, op.mesh.n_dof)
    _check(load().vfd_apply_parts(op.handle, int(parts), _ptr(X), _ptr(Y), nrhs, ld, _stream(stream)))
    return Y


def vfd_apply_noalloc(op, X, Y, stream=None):
    """Y = A X with no allocation inside the call (X, Y on the device)."""
    nrhs, ld = _nrhs_ld(X, op.mesh.n_dof)
    _check(load().vfd_apply_noalloc(op.handle, _ptr(X), _ptr(Y), nrhs, ld, _stream(stream)))
    return Y


def vfd_grad(op, U, Lam, g_s, g_logk, stream=None):
    """g_s, g_logk (device, n_vert) = -sum_r Lam_r^T (dA/dtheta) U_r for nodal fields."""
    nrhs, ld = _nrhs_ld(U, op.mesh.n_dof)
    _check(load().vfd_grad(op.handle, _ptr(U), _ptr(Lam), nrhs, ld, _ptr(g_s), _ptr(g_logk), _stream(stream)))
    return g_s, g_logk


def vfd_solve(op, F, U, rtol=1e-10, max_it=10000, stream=None, raise_on_noconv=False):
    """Returns (status, iters[nrhs], relres[nrhs]); U is updated in place."""
    nrhs, ld = _nrhs_ld(F, op.mesh.n_dof)
    it = (C.c_int * nrhs)()
    rr = np.zeros(nrhs)
    st = load().vfd_solve(op.handle, _ptr(F), _ptr(U), nrhs, ld, float(rtol), int(max_it), it,
                          rr.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream))
    if st not in (VFD_OK, VFD_ENOCONV) or (raise_on_noconv and st != VFD_OK):
        _check(st)
    return st, np.array(list(it)), rr


class Batch:
    """A batch of VFD_FP32 / VFD_BF16 operators (keeps them alive)."""

    def __init__(self, handle, ops):
        self.handle = handle
        self.ops = list(ops)

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().vfd_batch_free(self.handle)
            except Exception:
                pass
            self.handle = None


def vfd_batch_create(ops):
    arr = (C.c_void_p * len(ops))(*[op.handle for op in ops])
    h = C.c_void_p()
    _check(load().vfd_batch_create(arr, len(ops), C.byref(h)))
    return Batch(h, ops)


def _blocks(batch, Xs):
    ptrs = (C.c_void_p * len(Xs))(*[a.data_ptr() for a in Xs])
    lds = (C.c_int64 * len(Xs))(*[int(a.shape[1]) for a in Xs])
    nrhs = int(Xs[0].shape[0])
    for a, op in zip(Xs, batch.ops):
        if a.ndim != 2 or a.shape[0] != nrhs or a.shape[1] != op.mesh.n_dof:
            raise ValueError("batch blocks must be (nrhs, n_dof) tensors, one per operator")
    return ptrs, lds, nrhs


def vfd_batch_apply(batch, Xs, Ys, stream=None):
    """Ys[m] = A_low,m Xs[m]; Xs, Ys: lists of (nrhs, n_dof(m)) float64 CUDA tensors, nrhs % 64 == 0."""
    xp, lds, nrhs = _blocks(batch, Xs)
    yp, _, _ = _blocks(batch, Ys)
    _check(load().vfd_batch_apply(batch.handle, xp, yp, lds, nrhs, _stream(stream)))
    return Ys


def vfd_batch_solve(batch, Fs, Us, rtol=1e-8, max_it=100000, stream=None, raise_on_noconv=False):
    """Batched mixed-precision solve (CG with FP64 reliable updates); returns
    (status, iters (nmesh, nrhs), relres (nmesh, nrhs))."""
    fp, lds, nrhs = _blocks(batch, Fs)
    up, _, _ = _blocks(batch, Us)
    n = len(Fs) * nrhs
    it = (C.c_int * n)()
    rr = np.zeros(n)
    st = load().vfd_batch_solve(batch.handle, fp, up, lds, nrhs, float(rtol), int(max_it), it,
                                rr.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream))
    if st not in (VFD_OK, VFD_ENOCONV) or (raise_on_noconv and st != VFD_OK):
        _check(st)
    return st, np.array(list(it)).reshape(len(Fs), nrhs), rr.reshape(len(Fs), nrhs)


def vfd_batch_tuning(batch):
    """(chosen (stage columns, depth, split, warps, accumulator sets, tcgen05), candidate times in us) of
    the batch's near-panel kernel."""
    ch = (C.c_int * 6)()
    us = (C.c_float * 32)()
    nc = C.c_int()
    _check(load().vfd_batch_tuning(batch.handle, ch, us, 32, C.byref(nc)))
    return tuple(ch), list(us)[:nc.value]


def vfd_batch_set_config(batch, cfg):
    """Pin the near-panel candidate cfg (or -1: time them all); returns the number of candidates."""
    n = C.c_int()
    _check(load().vfd_batch_set_config(batch.handle, int(cfg), C.byref(n)))
    return n.value


def vfd_batch_set_wait_limit(batch, seconds):
    """Bound (seconds) of the tensor-core kernel's device waits; 0 = give up at once."""
    _check(load().vfd_batch_set_wait_limit(batch.handle, float(seconds)))


def vfd_batch_set_update_drop(batch, drop):
    """Recursive-residual reduction (0 < drop < 1) between the batched solve's FP64 reliable updates."""
    _check(load().vfd_batch_set_update_drop(batch.handle, float(drop)))


def vfd_precondition(op, kind=VFD_PREC_TWO_LEVEL, stream=None):
    """Preconditioner of the op's CG solves: FP64 CG and the batched mixed-precision
    solve (VFD_PREC_TWO_LEVEL, VFD_PREC_BLOCK_JACOBI; VFD_PREC_NONE: plain CG)."""
    _check(load().vfd_precondition(op.handle, int(kind), _stream(stream)))


def vfd_load(mesh, f_nodal, F, stream=None):
    _check(load().vfd_load(mesh.handle, _ptr(f_nodal), _ptr(F), _stream(stream)))
    return F


def vfd_op_rho(op, rho, stream=None):
    _check(load().vfd_op_rho(op.handle, _ptr(rho), _stream(stream)))
    return rho


def vfd_op_timings(op):
    """Device milliseconds per assembly phase (needs flags=VFD_ASSEMBLE_TIMED)."""
    a = np.zeros(len(TIMING_KEYS))
    _check(load().vfd_op_timings(op.handle, a.ctypes.data_as(C.POINTER(C.c_double)), len(a)))
    return dict(zip(TIMING_KEYS, a.tolist()))


def vfd_op_far_ranks(op):
    """Rank of every far level of the FP64 far field, coarsest first (after
    recompression the padded per-level ranks)."""
    nl = C.c_int()
    _check(load().vfd_op_far_ranks(op.handle, None, 0, C.byref(nl)))
    r = (C.c_int * max(nl.value, 1))()
    _check(load().vfd_op_far_ranks(op.handle, r, nl.value, C.byref(nl)))
    return [int(r[i]) for i in range(nl.value)]


def vfd_selftest_math(mesh, which, x, out, stream=None):
    """out = log(x) (which=0), exp(x) (which=1), cos(pi x) (which=2) or
    sin(pi x) (which=3) by the library's table-driven FP64 routines (device
    tensors)."""
    _check(load().vfd_selftest_math(mesh.handle, int(which), x.numel(), _ptr(x), _ptr(out), _stream(stream)))
    return out


def vfd_free_op(op):
    if op.handle:
        load().vfd_free_op(op.handle)
        op.handle = None


def vfd_free_mesh(mesh):
    if mesh.handle:
        load().vfd_free_mesh(mesh.handle)
        mesh.handle = None


def vfd_last_error():
    return load().vfd_last_error().decode()
