"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only *generates inputs*: simplicial meshes of the shapes used in the
paper's experiments (Sec. 7: unit disk with an annulus out to R, the square
(-2,2)^2 around (-1,1)^2, and the 1D interval analogue), descriptors of the
fractional-order field s(x) and of log kappa(x), and right-hand sides.  It
holds none of the method's arithmetic (no quadrature, no kernel, no
assembly); both the oracle and the CUDA path evaluate the field descriptors
with their own code.

Every generator is deterministic in its integer seed (numpy PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field as dc_field
from typing import Optional

import numpy as np

__all__ = [
    "Mesh", "Field", "interval_mesh", "disk_mesh", "square_mesh", "square_mesh_graded", "graded_coordinates",
    "disk_mesh_for_dofs", "square_mesh_for_dofs", "const_field", "fourier_field",
    "random_fourier_field", "config2_s_field", "sigmoid_field", "gauss_bump_field",
    "tensor_bump_field", "nodal_field", "frac_laplacian_const", "closed_form_u",
    "rhs_vectors", "workload", "ball_workload", "kuhn_ball_mesh",
]


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------
@dataclass
class Mesh:
    """A conforming simplicial mesh of Omega = Omega_i U Omega_e.

    coords: (M, d) float64 vertex coordinates.
    cells:  (C, d+1) int32 vertex indices.
    cell_is_interior: (C,) uint8, 1 for cells of Omega_i, 0 for Omega_e.
    """
    d: int
    coords: np.ndarray
    cells: np.ndarray
    cell_is_interior: np.ndarray
    name: str = ""
    meta: dict = dc_field(default_factory=dict)

    @property
    def n_vert(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_cell(self) -> int:
        return int(self.cells.shape[0])


def interval_mesh(n_interior: int, R: float = 1.1) -> Mesh:
    """Uniform P1 mesh of (-R, R) with Omega_i = (-1, 1).

    n_interior nodes strictly inside (-1,1), spacing h = 2/(n_interior+1); the
    exterior (-R,-1) U (1,R) is cut into ceil((R-1)/h) equal cells per side so
    that the mesh ends exactly at +-R (needed by the exterior tail formula).
    """
    h = 2.0 / (n_interior + 1)
    inner = -1.0 + h * np.arange(n_interior + 2)
    inner[-1] = 1.0
    n_ext = int(math.ceil((R - 1.0) / h - 1e-12))
    he = (R - 1.0) / n_ext
    right = 1.0 + he * np.arange(1, n_ext + 1)
    right[-1] = R
    left = -right[::-1]
    x = np.concatenate([left, inner, right])
    cells = np.stack([np.arange(len(x) - 1), np.arange(1, len(x))], axis=1).astype(np.int32)
    mid = 0.5 * (x[cells[:, 0]] + x[cells[:, 1]])
    is_int = (np.abs(mid) < 1.0).astype(np.uint8)
    return Mesh(1, x.reshape(-1, 1).astype(np.float64), cells, is_int,
                name=f"interval_N{n_interior}", meta={"h": h, "R": R})


def _ring_zip(inner_ids, outer_ids):
    """Triangles between two concentric rings whose nodes sit at equally spaced
    angles starting at 0 (topology only)."""
    n1, n2 = len(inner_ids), len(outer_ids)
    tris = []
    i = j = 0
    while i < n1 or j < n2:
        a_next = (i + 1) / n1 if i < n1 else 2.0
        b_next = (j + 1) / n2 if j < n2 else 2.0
        if i < n1 and (j >= n2 or a_next < b_next):
            tris.append((inner_ids[i], inner_ids[(i + 1) % n1], outer_ids[j % n2]))
            i += 1
        else:
            tris.append((inner_ids[i % n1], outer_ids[(j + 1) % n2], outer_ids[j]))
            j += 1
    return tris


def _orient(coords, cells):
    p0, p1, p2 = coords[cells[:, 0]], coords[cells[:, 1]], coords[cells[:, 2]]
    det = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])
    neg = det < 0
    cells[neg, 1], cells[neg, 2] = cells[neg, 2].copy(), cells[neg, 1].copy()
    return cells


def disk_mesh(K: int, R: float = 1.1, jitter: float = 0.2, seed: int = 0,
              n_ext: Optional[int] = None) -> Mesh:
    """Quasi-uniform triangle mesh of the disk of radius R, Omega_i = unit disk.

    Concentric rings: ring k (k=1..K) at radius k/K carries 6k nodes; ring K is
    the circle r=1.  The annulus 1<r<R carries n_ext further rings (default
    round((R-1)K)), ring K+j at radius 1 + j (R-1)/n_ext with 6(K+j) nodes.
    Seeded jitter of at most `jitter`*h moves every node that is not on r=1 or
    r=R isotropically; nodes on those two circles move only along the circle.
    """
    rng = np.random.default_rng(seed)
    h = 1.0 / K
    if n_ext is None:
        n_ext = max(1, int(round((R - 1.0) * K)))
    radii = [k * h for k in range(K + 1)] + [1.0 + j * (R - 1.0) / n_ext for j in range(1, n_ext + 1)]
    radii[K] = 1.0
    radii[-1] = R
    coords = [(0.0, 0.0)]
    ring_ids = [[0]]
    ring_of = [0]
    for k in range(1, len(radii)):
        n = 6 * k
        ids = list(range(len(coords), len(coords) + n))
        th = 2.0 * math.pi * np.arange(n) / n
        for t in th:
            coords.append((radii[k] * math.cos(t), radii[k] * math.sin(t)))
            ring_of.append(k)
        ring_ids.append(ids)
    coords = np.array(coords, dtype=np.float64)
    ring_of = np.array(ring_of)
    tris = [(0, ring_ids[1][j], ring_ids[1][(j + 1) % 6]) for j in range(6)]
    for k in range(1, len(radii) - 1):
        tris += _ring_zip(ring_ids[k], ring_ids[k + 1])
    cells = np.array(tris, dtype=np.int32)
    # interior cells: all vertices on rings <= K
    is_int = (ring_of[cells].max(axis=1) <= K).astype(np.uint8)
    # jitter
    if jitter > 0:
        M = coords.shape[0]
        on_circle = (ring_of == K) | (ring_of == len(radii) - 1)
        u = rng.random(M)
        v = rng.random(M)
        w = rng.random(M)
        rad = jitter * h * np.sqrt(u)
        ang = 2.0 * math.pi * v
        disp = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
        disp[on_circle] = 0.0
        coords = coords + disp
        # tangential move on the two circles
        idx = np.nonzero(on_circle)[0]
        r = np.hypot(coords[idx, 0], coords[idx, 1])
        th = np.arctan2(coords[idx, 1], coords[idx, 0]) + jitter * h * (2 * w[idx] - 1) / r
        coords[idx, 0] = r * np.cos(th)
        coords[idx, 1] = r * np.sin(th)
    cells = _orient(coords, cells)
    return Mesh(2, coords, cells, is_int, name=f"disk_K{K}",
                meta={"h": h, "R": R, "K": K, "n_ext": n_ext, "seed": seed})


def disk_mesh_for_dofs(n_dofs: int, R: float = 1.1, jitter: float = 0.2, seed: int = 0) -> Mesh:
    """Disk mesh whose interior DoF count 1 + 3K(K-1) is closest to n_dofs."""
    K = max(2, int(round(0.5 + math.sqrt(max(n_dofs - 1, 0) / 3.0 + 0.25))))
    return disk_mesh(K, R=R, jitter=jitter, seed=seed)


def square_mesh(mc: int, jitter: float = 0.0, seed: int = 0) -> Mesh:
    """Uniform triangulation of Omega = (-2,2)^2 with Omega_i = (-1,1)^2.

    mc (even) cells per side of Omega_i, 2*mc per side of Omega, each square
    cut along its (+1,+1) diagonal.  mc = 2^(j+1) gives the paper's mesh T_j
    with leg 2^-j (h_j = sqrt(2)/2^j): T_6 (mc=128) has 127^2 = 16129 interior
    DoFs and 2*256^2 = 131072 cells.  Optional seeded jitter moves a node coordinate
    only when that coordinate is not on one of the lines -2,-1,1,2, so the
    boundaries of Omega and Omega_i stay straight.
    """
    assert mc % 2 == 0
    n = 2 * mc
    hl = 4.0 / n
    g = -2.0 + hl * np.arange(n + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    vid = lambda i, j: j * (n + 1) + i
    cells = []
    is_int = []
    for j in range(n):
        for i in range(n):
            a, b, c, e = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            cells.append((a, b, c))
            cells.append((a, c, e))
            cx, cy = g[i] + 0.5 * hl, g[j] + 0.5 * hl
            inside = 1 if (abs(cx) < 1.0 and abs(cy) < 1.0) else 0
            is_int += [inside, inside]
    cells = np.array(cells, dtype=np.int32)
    is_int = np.array(is_int, dtype=np.uint8)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        d = jitter * hl * (2 * rng.random(coords.shape) - 1)
        fixed = np.zeros_like(coords, dtype=bool)
        for L in (-2.0, -1.0, 1.0, 2.0):
            fixed |= np.abs(coords - L) < 1e-12
        d[fixed] = 0.0
        coords = coords + d
    cells = _orient(coords, cells)
    return Mesh(2, coords, cells, is_int, name=f"square_mc{mc}",
                meta={"h": hl, "mc": mc, "seed": seed})


def graded_coordinates(mc: int, grade: float) -> np.ndarray:
    """1D nodes of [-2, 2]: mc equal cells on [-1, 1] (spacing h = 2/mc), and on
    each side of it cells growing geometrically by the factor `grade` from h*grade
    until the side's length 1 is filled; the outer cells are scaled by a common
    factor so that the last node is exactly at +-2 (the ratio stays `grade`)."""
    h = 2.0 / mc
    sp = []
    tot = 0.0
    while tot < 1.0 - 1e-12:
        sp.append(h * grade ** (len(sp) + 1))
        tot += sp[-1]
    sp = np.array(sp) / tot          # spacings of one side, summing to 1
    inner = -1.0 + h * np.arange(mc + 1)
    inner[-1] = 1.0
    right = 1.0 + np.cumsum(sp)
    right[-1] = 2.0
    return np.concatenate([-right[::-1], inner, right])


def square_mesh_graded(mc: int, grade: float = 1.5) -> Mesh:
    """Triangulation of Omega = (-2,2)^2 with Omega_i = (-1,1)^2 whose exterior
    is graded: the tensor grid of graded_coordinates(mc, grade) in x and y,
    each rectangle cut along its (+1,+1) diagonal.  Omega_i is meshed exactly as
    by square_mesh(mc) (the same (mc-1)^2 interior DoFs); the exterior cells
    grow geometrically away from the interface (the remark of Sec. 7.2 on the
    cost of M with a quasi-uniform exterior)."""
    assert mc % 2 == 0 and grade >= 1.0
    g = graded_coordinates(mc, grade)
    n = len(g) - 1
    X, Y = np.meshgrid(g, g, indexing="xy")
    coords = np.stack([X.ravel(), Y.ravel()], axis=1)
    I, J = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    I, J = I.ravel(), J.ravel()
    a, b, c, e = J * (n + 1) + I, J * (n + 1) + I + 1, (J + 1) * (n + 1) + I + 1, (J + 1) * (n + 1) + I
    cells = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, e], 1)], axis=0).astype(np.int32)
    cx = 0.5 * (g[I] + g[I + 1])
    cy = 0.5 * (g[J] + g[J + 1])
    inside = ((np.abs(cx) < 1.0) & (np.abs(cy) < 1.0)).astype(np.uint8)
    is_int = np.concatenate([inside, inside])
    cells = _orient(coords, cells)
    return Mesh(2, coords, cells, is_int, name=f"square_graded_mc{mc}_g{grade:g}",
                meta={"h": 2.0 / mc, "mc": mc, "grade": grade})


def square_mesh_for_dofs(n_dofs: int, jitter: float = 0.2, seed: int = 0) -> Mesh:
    """Square mesh whose interior DoF count (mc-1)^2 is closest to n_dofs."""
    mc = int(round(math.sqrt(n_dofs))) + 1
    if mc % 2:
        mc += 1
    return square_mesh(mc, jitter=jitter, seed=seed)


# ----------------------------------------------------------------------------
# field descriptors
# ----------------------------------------------------------------------------
def kuhn_ball_mesh(n: int, L: float = 1.1, R_in: float = 1.0, R_out: float = 1.1) -> Mesh:
    """Tetrahedral mesh of a ball: the cube [-L, L]^3 cut into n^3 cubes, each
    cube into the 6 Kuhn tetrahedra around its main diagonal (conforming
    across cubes); cells whose centroid lies in |c| < R_out are kept (Omega),
    those with |c| < R_in are interior (Omega_i, a polytope approximating the
    unit ball).  Vertices are renumbered to the ones used; every tetrahedron
    has positive orientation."""
    h = 2.0 * L / n
    g = np.arange(n + 1) * h - L
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(i, j, k):
        return (i * (n + 1) + j) * (n + 1) + k

    # the 6 monotone lattice paths from (0,0,0) to (1,1,1)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    cells = []
    for p in perms:
        o = np.zeros((len(I), 3), dtype=np.int64)
        vs = [vid(I, J, K)]
        for ax in p:
            o[:, ax] += 1
            vs.append(vid(I + o[:, 0], J + o[:, 1], K + o[:, 2]))
        cells.append(np.stack(vs, axis=1))
    cells = np.concatenate(cells, axis=0)
    cen = coords[cells].mean(axis=1)
    r = np.linalg.norm(cen, axis=1)
    keep = r < R_out
    cells, r = cells[keep], r[keep]
    inter = (r < R_in).astype(np.uint8)
    used = np.unique(cells)
    remap = -np.ones(len(coords), dtype=np.int64)
    remap[used] = np.arange(len(used))
    coords = coords[used]
    cells = remap[cells]
    # positive orientation
    P = coords[cells]
    det = np.einsum("ij,ij->i", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))
    neg = det < 0
    cells[neg, 2], cells[neg, 3] = cells[neg, 3].copy(), cells[neg, 2].copy()
    return Mesh(3, coords.astype(np.float64), cells.astype(np.int32), inter, name=f"kuhn_ball_{n}",
                meta={"L": L, "R_in": R_in, "R_out": R_out, "h": h})


@dataclass
class Field:
    """A scalar field on R^d, value = squash(c0 + sum of terms).

    fourier rows (k1,k2,k3, amp, phase): amp*cos(pi*(k.x) + phase), integer k.
    gauss rows (x0,y0,z0, amp, c):       amp*exp(-c*|x-x0|^2).
    tbump rows (x0,y0,z0, amp, ell):     amp*prod_i bump(x_i - x0_i; ell),
        bump(t; ell) = exp(-1/(1-r^2)) for r = 2t/ell, |r|<1, else 0.
    squash: 0 none; 1 lo + (hi-lo)/(1+exp(-v)).
    nodal: optional array of values at the mesh vertices (P1 field); when set
    the other members are ignored.
    """
    c0: float = 0.0
    fourier: np.ndarray = dc_field(default_factory=lambda: np.zeros((0, 5)))
    gauss: np.ndarray = dc_field(default_factory=lambda: np.zeros((0, 5)))
    tbump: np.ndarray = dc_field(default_factory=lambda: np.zeros((0, 5)))
    squash: int = 0
    lo: float = 0.0
    hi: float = 1.0
    nodal: Optional[np.ndarray] = None

    @property
    def is_const(self) -> bool:
        return (self.nodal is None and len(self.fourier) == 0 and len(self.gauss) == 0
                and len(self.tbump) == 0)


def const_field(v: float) -> Field:
    return Field(c0=float(v))


def fourier_field(c0, rows) -> Field:
    rows = np.asarray(rows, dtype=np.float64).reshape(-1, 5)
    assert np.all(rows[:, :3] == np.round(rows[:, :3])), "wavevectors must be integer"
    return Field(c0=float(c0), fourier=rows)


def random_fourier_field(seed: int, sigma: float, d: int = 2, n_modes: int = 16,
                         kmax: int = 3, mean: float = 0.0) -> Field:
    """16 cosine modes with integer wavevectors 1 <= |k|_inf <= kmax, normal
    amplitudes, uniform phases, scaled so the pointwise std is sigma."""
    rng = np.random.default_rng(seed)
    rows = []
    while len(rows) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=d)
        if np.max(np.abs(k)) < 1:
            continue
        kk = np.zeros(3)
        kk[:d] = k
        rows.append([kk[0], kk[1], kk[2], rng.standard_normal(), 2 * math.pi * rng.random()])
    rows = np.array(rows)
    rows[:, 3] *= sigma / math.sqrt(0.5 * np.sum(rows[:, 3] ** 2))
    return Field(c0=mean, fourier=rows)


def config2_s_field() -> Field:
    """s(x) = 0.25 + 0.5(0.5 + 0.5 sin(2 pi x1) cos(2 pi x2)), written as
    0.5 + 0.125 cos(pi(2,2).x - pi/2) + 0.125 cos(pi(2,-2).x - pi/2)."""
    return fourier_field(0.5, [[2, 2, 0, 0.125, -math.pi / 2], [2, -2, 0, 0.125, -math.pi / 2]])


def sigmoid_field(base: Field, lo: float, hi: float) -> Field:
    return Field(c0=base.c0, fourier=base.fourier, gauss=base.gauss, tbump=base.tbump,
                 squash=1, lo=lo, hi=hi)


def gauss_bump_field(c0, x0, amp, c) -> Field:
    x0 = list(x0) + [0.0] * (3 - len(x0))
    return Field(c0=float(c0), gauss=np.array([[x0[0], x0[1], x0[2], amp, c]], dtype=np.float64))


def tensor_bump_field(c0, xc, amp, ell) -> Field:
    xc = list(xc) + [0.0] * (3 - len(xc))
    return Field(c0=float(c0), tbump=np.array([[xc[0], xc[1], xc[2], amp, ell]], dtype=np.float64))


def nodal_field(values) -> Field:
    return Field(nodal=np.ascontiguousarray(values, dtype=np.float64))


# ----------------------------------------------------------------------------
# problem data
# ----------------------------------------------------------------------------
def frac_laplacian_const(d: int, s: float) -> float:
    """C_{d,s} = 2^{2s} s Gamma(s + d/2) / (pi^{d/2} Gamma(1-s)), the constant of
    the integral fractional Laplacian; the diffusion coefficient a = C_{d,s}/2
    makes the bilinear form equal to ((-Delta)^s u, v)."""
    return 2.0 ** (2 * s) * s * math.gamma(s + d / 2.0) / (math.pi ** (d / 2.0) * math.gamma(1.0 - s))


def closed_form_u(x: np.ndarray, d: int, s: float) -> np.ndarray:
    """Solution of (-Delta)^s u = 1 in the unit ball, u = 0 outside:
    u = 2^{-2s} Gamma(d/2) / (Gamma(d/2+s) Gamma(1+s)) (1-|x|^2)_+^s."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, d)
    c = 2.0 ** (-2 * s) * math.gamma(d / 2.0) / (math.gamma(d / 2.0 + s) * math.gamma(1.0 + s))
    r2 = np.sum(x * x, axis=1)
    return c * np.maximum(1.0 - r2, 0.0) ** s


def rhs_vectors(n: int, nrhs: int, seed: int) -> np.ndarray:
    """(n, nrhs) column-major-ready float64 N(0,1) white noise."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, nrhs)))


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
def batch_workload(n_mesh: int = 24, n_min: int = 2000, ratio: float = 65.0, seed0: int = 3000):
    """Many meshes of uneven size: mesh i (i = 0..n_mesh-1) targets
    round(n_min * ratio^(i/(n_mesh-1))) interior DoFs (log-uniform sizes, 2k to
    130k for the defaults); even i: the square (-1,1)^2 inside (-2,2)^2, odd i:
    the unit disk with an annulus to R = 1.1; jitter 0.2 of the local spacing.
    Fields per mesh: s = 0.1 + 0.8 sigmoid(F_a) with F_a a seeded 16-mode
    Fourier field (sigma 1), log kappa a seeded Fourier field (sigma 0.5).
    Returns a list of (mesh, s_field, logkappa_field, target_dofs)."""
    out = []
    for i in range(n_mesh):
        n = int(round(n_min * ratio ** (i / max(n_mesh - 1, 1))))
        seed = seed0 + i
        m = square_mesh_for_dofs(n, jitter=0.2, seed=seed) if i % 2 == 0 else \
            disk_mesh_for_dofs(n, R=1.1, jitter=0.2, seed=seed)
        s = sigmoid_field(random_fourier_field(seed + 100, 1.0), 0.1, 0.9)
        k = random_fourier_field(seed + 200, 0.5)
        out.append((m, s, k, n))
    return out


def ball_workload(n: int, seed: int = 5000):
    """The 3D configuration: the Kuhn-grid ball kuhn_ball_mesh(n) (spacing
    2.2/n; Omega_i the cells with centroid inside the unit ball, Omega those
    inside radius 1.1), s = 0.2 + 0.6 exp(-4 |x - x0|^2) with x0 seeded uniform
    in the ball of radius 0.5, log kappa a seeded 3D Fourier field (sigma 0.5).
    Returns (mesh, s_field, logkappa_field, params)."""
    rng = np.random.default_rng(seed)
    while True:
        x0 = rng.uniform(-0.5, 0.5, 3)
        if np.linalg.norm(x0) < 0.5:
            break
    m = kuhn_ball_mesh(n)
    s = gauss_bump_field(0.2, x0, 0.6, 4.0)
    k = random_fourier_field(seed + 1, 0.5, d=3)
    return m, s, k, dict(s_bar=0.9, tail=0, R=1.1, leaf=64, p=4, lam=0.75, x0=x0.tolist())


def workload(name: str):
    """Named synthetic workloads: returns (mesh, s_field, logkappa_field, params).

    'interval512': 1D (-1,1), 512 interior nodes, s=0.3, a=C_{1,0.3}/2, zero
                   volume condition on R \\ (-1,1) (tail), s_bar = 0.3.
    'disk33k':     2D unit disk + annulus to R=1.1, K=96 rings (34k vertices),
                   s = 0.25+0.5(0.5+0.5 sin(2 pi x1)cos(2 pi x2)), log a a seeded
                   Fourier field with sigma=0.5, s_bar=0.9, leaf 64, lambda 0.75,
                   Chebyshev p=8 (rank 64): an interpolation order at which the
                   far field meets the matvec tolerance 1e-6 on this disk with a
                   margin (about 1e-7); the low-precision inner operator of the
                   batched solves uses p=4.
    'disk33k_r16': the same disk and fields with p=4 (rank 16).
    'disk_small':  same fields on a K=12 disk (parity-size).
    'disk130k':    the same fields on a K=208 disk (~130k DoFs, rank 64): panels
                   larger than the 129 MB L2 (profiling captures of the
                   near-panel kernels).
    """
    if name == "interval512":
        s = 0.3
        m = interval_mesh(512, R=1.1)
        return m, const_field(s), const_field(math.log(frac_laplacian_const(1, s) / 2)), \
            dict(s_bar=0.3, tail=1, R=1.1, leaf=64, p=4)
    if name.startswith("disk"):
        K, p = {"disk33k": (96, 8), "disk33k_r16": (96, 4), "disk_small": (12, 4), "disk_medium": (30, 4),
                "disk130k": (208, 8)}[name]
        m = disk_mesh(K, R=1.1, jitter=0.2, seed=2000 + K)
        return m, config2_s_field(), random_fourier_field(2001, 0.5), \
            dict(s_bar=0.9, tail=0, R=1.1, leaf=64, p=p, lam=0.75, inner_p=min(p, 4))
    raise KeyError(name)
