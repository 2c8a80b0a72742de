"""Graded exterior meshes (the remark of Sec. 7.2: with a quasi-uniform exterior
the weighted mass matrix M, whose density integrates the kernel over the
exterior, dominates the assembly of the square problem).  The graded square
keeps the interior mesh of the quasi-uniform one and lets the exterior cells
grow geometrically away from the interface.

* structure: the same interior DoFs as square_mesh(mc), far fewer exterior
  cells, a conforming triangulation of (-2,2)^2 whose outer nodes are at +-2,
  spacing ratio `grade` between neighbouring exterior cells;
* the discrete operator stays SPD and the solution with f = 1 differs from
  the quasi-uniform one by far less than the discretisation error (both
  approximate the same problem; the exterior only enters through the density
  of M and the touching pairs of B).
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("mc,grade", [(8, 1.5), (16, 1.3), (128, 1.5)])
def test_graded_square_structure(mc, grade):
    g = synth.graded_coordinates(mc, grade)
    assert g[0] == -2.0 and g[-1] == 2.0 and np.all(np.diff(g) > 0)
    h = 2.0 / mc
    inner = g[(g > -1 - 1e-12) & (g < 1 + 1e-12)]
    assert len(inner) == mc + 1 and np.allclose(np.diff(inner), h)
    right = np.diff(g[g >= 1.0 - 1e-12])
    assert np.allclose(right[1:] / right[:-1], grade)
    m = synth.square_mesh_graded(mc, grade)
    u = synth.square_mesh(mc)
    assert int(m.cell_is_interior.sum()) == int(u.cell_is_interior.sum())
    assert m.n_cell - int(m.cell_is_interior.sum()) < (0.5 if mc >= 16 else 1.0) * (u.n_cell - int(u.cell_is_interior.sum()))
    dof, N = oracle.dofs(m)
    assert N == (mc - 1) ** 2
    # conforming: every edge in one cell (on the outer boundary) or two
    e = np.sort(np.concatenate([m.cells[:, [0, 1]], m.cells[:, [1, 2]], m.cells[:, [0, 2]]]), axis=1)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    assert cnt.max() == 2
    on_bd = np.all(np.abs(np.abs(m.coords[uniq[cnt == 1]]) - 2.0).min(axis=2) < 1e-12, axis=1) | \
        np.any(np.all(np.abs(np.abs(m.coords[uniq[cnt == 1]]) - 2.0) < 1e-12, axis=1), axis=1)
    assert on_bd.all()
    P = m.coords[m.cells]
    area = 0.5 * ((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                  (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    assert np.all(area > 0) and abs(area.sum() - 16.0) < 1e-10


@pytest.mark.parametrize("mc", [8, 12])
def test_graded_exterior_keeps_the_solution(mc):
    s, k = synth.const_field(0.5), synth.const_field(0.0)
    sol = {}
    for name, m in (("uniform", synth.square_mesh(mc)), ("graded", synth.square_mesh_graded(mc, 1.5))):
        A = oracle.assemble(m, s, k, s_bar=0.9, n_sing=3)
        assert np.allclose(A.A, A.A.T, rtol=0, atol=1e-13 * np.abs(A.A).max())
        np.linalg.cholesky(A.A)
        F = oracle.load(m, np.ones(m.n_vert))
        U = oracle.cholesky_solve(A.A, F)
        inner = np.abs(m.coords).max(axis=1) < 1.0 - 1e-9
        order = np.lexsort((m.coords[inner, 0], m.coords[inner, 1]))
        u = np.zeros(m.n_vert)
        u[A.dof >= 0] = U[A.dof[A.dof >= 0]]
        sol[name] = u[inner][order]
    d = np.linalg.norm(sol["graded"] - sol["uniform"]) / np.linalg.norm(sol["uniform"])
    assert d < 2e-3, d
