"""CPU oracle for the variable-order fractional FE operator (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py; never by the product package.  It shares no code
with the CUDA path.  The arithmetic lives in vfd_oracle.c (plain C, FP64,
OpenMP); this module compiles it with gcc and marshals numpy arrays.

Every function cites the passage of the paper it follows; see vfd_oracle.c.
Parity status: all routines are pinned by tests/test_oracle_*.py (closed
forms, invariants, special cases and brute-force quadrature).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vfd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (-O2 -fopenmp)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        up = C.POINTER(C.c_ubyte)
        L.oracle_gauss01.argtypes = [C.c_int, dp, dp]
        L.oracle_dofs.argtypes = [C.c_int, C.c_int, C.c_int, ip, up, ip]
        L.oracle_dofs.restype = C.c_int
        L.oracle_assemble.argtypes = [C.c_int, C.c_int, C.c_int, dp, ip, up, dp, dp, dp, dp, dp,
                                      dp, dp, dp, dp, dp]
        L.oracle_assemble.restype = C.c_int
        L.oracle_pair_local.argtypes = [C.c_int, C.c_int, dp, dp, ip, ip, dp, dp, dp, dp,
                                        C.c_double, C.c_int, dp]
        L.oracle_pair_local.restype = C.c_int
        L.oracle_tail.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double]
        L.oracle_tail.restype = C.c_double
        L.oracle_load.argtypes = [C.c_int, C.c_int, C.c_int, dp, ip, up, dp, dp]
        L.oracle_load.restype = C.c_int
        L.oracle_cholesky_solve.argtypes = [C.c_int, dp, dp, dp]
        L.oracle_cholesky_solve.restype = C.c_int
        L.oracle_field.argtypes = [C.c_int, dp, dp]
        L.oracle_field.restype = C.c_double
        L.oracle_gamma.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double]
        L.oracle_gamma.restype = C.c_double
        L.oracle_num_threads.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_set_threads.restype = None
        L.oracle_cg.argtypes = [C.c_int, dp, dp, dp, C.c_double, C.c_int]
        L.oracle_cg.restype = C.c_int
        L.oracle_grad.argtypes = [C.c_int, C.c_int, C.c_int, dp, ip, up, dp, dp, dp, C.c_int, dp, dp, dp, dp]
        L.oracle_grad.restype = C.c_int
        L.oracle_apply_rows.argtypes = [C.c_int, C.c_int, C.c_int, dp, ip, up, dp, dp, dp, dp, dp, dp, C.c_int,
                                        ip, dp]
        L.oracle_apply_rows.restype = C.c_int
        _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _up(a):
    return a.ctypes.data_as(C.POINTER(C.c_ubyte))


def field_desc(f):
    """Flatten a synth.Field into (descriptor, nodal) arrays for the C side."""
    hdr = [f.c0, len(f.fourier), len(f.gauss), len(f.tbump), f.squash, f.lo, f.hi]
    rows = [np.asarray(f.fourier, float).ravel(), np.asarray(f.gauss, float).ravel(),
            np.asarray(f.tbump, float).ravel()]
    desc = np.ascontiguousarray(np.concatenate([np.array(hdr, float)] + rows), dtype=np.float64)
    nodal = None if f.nodal is None else np.ascontiguousarray(f.nodal, dtype=np.float64)
    return desc, nodal


def gauss01(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().oracle_gauss01(n, _dp(x), _dp(w))
    return x, w


def dofs(mesh):
    """dof_of_vertex (-1 for non-DoF vertices) and N; DoFs numbered in
    increasing vertex order (Sec. 2.3: interior nodes first)."""
    T = np.ascontiguousarray(mesh.cells, dtype=np.int32)
    inn = np.ascontiguousarray(mesh.cell_is_interior, dtype=np.uint8)
    dof = np.zeros(mesh.n_vert, dtype=np.int32)
    N = lib().oracle_dofs(mesh.d, mesh.n_vert, mesh.n_cell, _ip(T), _up(inn), _ip(dof))
    return dof, N


class Assembled:
    """Dense FP64 results of the oracle: B, K, M (N x N), rho at interior
    quadrature points, optional route-1 Afull (M x M)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)

    @property
    def A(self):
        return self.B + self.K + self.M


def assemble(mesh, s, logk, s_bar=0.9, n_sing=3, tail=0, R=1.1, want_full=False):
    """Oracle assembly by the split B + K + M (route 2) and, if requested, by
    definition over all element pairs (route 1).  In 3D (tetrahedra) only the
    separated parts K, rho and M are assembled: the paper gives no singular
    rules for tetrahedron pairs, so B is returned as zeros (reading R20)."""
    L = lib()
    X = np.ascontiguousarray(mesh.coords, dtype=np.float64)
    T = np.ascontiguousarray(mesh.cells, dtype=np.int32)
    inn = np.ascontiguousarray(mesh.cell_is_interior, dtype=np.uint8)
    dof, N = dofs(mesh)
    sd, sn = field_desc(s)
    kd, kn = field_desc(logk)
    B = np.zeros((N, N))
    K = np.zeros((N, N))
    Mw = np.zeros((N, N))
    nq = 4 if mesh.d == 3 else 3   # element-rule points per cell (R3, R20)
    nqi = int(inn.sum()) * nq
    rho = np.zeros(nqi)
    Af = np.zeros((mesh.n_vert, mesh.n_vert)) if want_full else None
    params = np.array([s_bar, n_sing, tail, R], dtype=np.float64)
    t0 = time.perf_counter()
    n = L.oracle_assemble(mesh.d, mesh.n_vert, mesh.n_cell, _dp(X), _ip(T), _up(inn), _dp(sd), _dp(sn),
                          _dp(kd), _dp(kn), _dp(params), _dp(B), _dp(K), _dp(Mw), _dp(rho), _dp(Af))
    t1 = time.perf_counter()
    if n != N:
        raise RuntimeError("oracle_assemble failed")
    return Assembled(B=B, K=K, M=Mw, rho=rho, Afull=Af, dof=dof, N=N, seconds=t1 - t0)


def apply_rows(mesh, s, logk, x, rows, s_bar=0.9, n_sing=3, tail=0, R=1.1):
    """(A x)_i for the DoFs i in rows, A = B + K + M of the route-2 assembly
    without any approximation, one row at a time (O(|supp| |Q|) each): for
    sampled checks at sizes where the dense matrix does not fit."""
    X = np.ascontiguousarray(mesh.coords, dtype=np.float64)
    T = np.ascontiguousarray(mesh.cells, dtype=np.int32)
    inn = np.ascontiguousarray(mesh.cell_is_interior, dtype=np.uint8)
    sd, sn = field_desc(s)
    kd, kn = field_desc(logk)
    xv = np.ascontiguousarray(x, dtype=np.float64)
    rr = np.ascontiguousarray(rows, dtype=np.int32)
    y = np.zeros(len(rr))
    params = np.array([s_bar, n_sing, tail, R], dtype=np.float64)
    n = lib().oracle_apply_rows(mesh.d, mesh.n_vert, mesh.n_cell, _dp(X), _ip(T), _up(inn), _dp(sd), _dp(sn),
                                _dp(kd), _dp(kn), _dp(params), _dp(xv), len(rr), _ip(rr), _dp(y))
    if n < 0 or n != len(xv):
        raise ValueError("oracle_apply_rows: bad input")
    return y


def grad(mesh, s_nodal, logk_nodal, U, Lam, s_bar=0.9, n_sing=3):
    """g_s, g_logk (one entry per vertex) = -sum_r Lam_r^T (dA/dtheta) U_r for
    P1 (nodal) s and log kappa: the derivative of the route-2 matrix B + K + M
    term by term (kernel derivatives -ln|x-y| gamma and gamma/2 times the
    basis functions at both points), bounded exterior (no tail).  U, Lam:
    (N,) or (nrhs, N) in the DoF order of dofs()."""
    X = np.ascontiguousarray(mesh.coords, dtype=np.float64)
    T = np.ascontiguousarray(mesh.cells, dtype=np.int32)
    inn = np.ascontiguousarray(mesh.cell_is_interior, dtype=np.uint8)
    sn = np.ascontiguousarray(s_nodal, dtype=np.float64)
    kn = np.ascontiguousarray(logk_nodal, dtype=np.float64)
    U2 = np.ascontiguousarray(np.atleast_2d(U), dtype=np.float64)
    L2 = np.ascontiguousarray(np.atleast_2d(Lam), dtype=np.float64)
    gs = np.zeros(mesh.n_vert)
    gk = np.zeros(mesh.n_vert)
    params = np.array([s_bar, n_sing, 0, 0.0], dtype=np.float64)
    n = lib().oracle_grad(mesh.d, mesh.n_vert, mesh.n_cell, _dp(X), _ip(T), _up(inn), _dp(sn), _dp(kn),
                          _dp(params), U2.shape[0], _dp(U2), _dp(L2), _dp(gs), _dp(gk))
    if n < 0 or U2.shape[1] != n:
        raise ValueError("oracle_grad: bad input")
    return gs, gk


def pair_local(d, typ, P, Q, s, logk, s_bar, n_sing, pv=None, qv=None):
    """Local matrix of one touching pair (Sec. 4 singular rules); P, Q are the
    (d+1, d) reordered vertex coordinates of tau and tau'."""
    sd, sn = field_desc(s)
    kd, kn = field_desc(logk)
    P = np.ascontiguousarray(P, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    pv_ = None if pv is None else np.ascontiguousarray(pv, dtype=np.int32)
    qv_ = None if qv is None else np.ascontiguousarray(qv, dtype=np.int32)
    Lm = np.zeros(25)
    nl = lib().oracle_pair_local(d, typ, _dp(P), _dp(Q), None if pv_ is None else _ip(pv_),
                                 None if qv_ is None else _ip(qv_), _dp(sd), _dp(sn), _dp(kd), _dp(kn),
                                 float(s_bar), int(n_sing), _dp(Lm))
    if nl < 0:
        raise ValueError("bad n_sing")
    return Lm[:nl * nl].reshape(nl, nl)


def tail(d, x, s, a, R):
    x = np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)
    return lib().oracle_tail(d, _dp(x), float(s), float(a), float(R))


def load(mesh, f_nodal):
    """P1 load F = M0 f over interior cells (DoF order of dofs())."""
    X = np.ascontiguousarray(mesh.coords, dtype=np.float64)
    T = np.ascontiguousarray(mesh.cells, dtype=np.int32)
    inn = np.ascontiguousarray(mesh.cell_is_interior, dtype=np.uint8)
    f = np.ascontiguousarray(f_nodal, dtype=np.float64)
    _, N = dofs(mesh)
    F = np.zeros(N)
    lib().oracle_load(mesh.d, mesh.n_vert, mesh.n_cell, _dp(X), _ip(T), _up(inn), _dp(f), _dp(F))
    return F


def cholesky_solve(A, F):
    """Dense Cholesky solve (the oracle's own, not LAPACK)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    F = np.ascontiguousarray(F, dtype=np.float64)
    U = np.zeros_like(F)
    rc = lib().oracle_cholesky_solve(A.shape[0], _dp(A), _dp(F), _dp(U))
    if rc != 0:
        raise np.linalg.LinAlgError(f"matrix not positive definite at pivot {rc - 1}")
    return U


def cg(A, F, rtol=1e-10, max_it=100000):
    """Plain dense CG (the paper's solver) from zero; returns (U, iterations)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    U = np.zeros_like(F)
    it = lib().oracle_cg(A.shape[0], _dp(A), _dp(F), _dp(U), float(rtol), int(max_it))
    return U, it


def field(d, f, x):
    sd, _ = field_desc(f)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().oracle_field(d, _dp(sd), _dp(x))


def gamma(d, r, sx, sy, lkx, lky):
    return lib().oracle_gamma(d, r, sx, sy, lkx, lky)


def num_threads():
    return lib().oracle_num_threads()


def set_threads(n):
    """OpenMP threads of the following oracle calls (for timing baselines)."""
    lib().oracle_set_threads(int(n))


def quad_points(mesh):
    """Interior element-rule points in the oracle's rho order (interior cells
    by increasing id, then the 3 points whose dominant barycentric weight sits
    on stored vertex 0,1,2; 1D: Gauss points left to right)."""
    d = mesh.d
    out = []
    if d == 2:
        B = np.full((3, 3), 1.0 / 6.0)
        np.fill_diagonal(B, 2.0 / 3.0)
    else:
        g = 0.5 * np.sqrt(0.6)
        t = np.array([0.5 - g, 0.5, 0.5 + g])
        B = np.stack([1 - t, t], axis=1)
    for c in np.nonzero(mesh.cell_is_interior)[0]:
        V = mesh.coords[mesh.cells[c]]
        out.append(B @ V)
    return np.concatenate(out, axis=0)
