"""Pins for the oracle's singular quadrature (Sec. 4 of the paper) and its
Gauss rule, against references that do not use the paper's Duffy maps:

* kernels that are polynomials (|x-y|^2, and 1) where the Sec. 4 rules with
  the matching s_bar are exact, compared with a high-order product rule;
* the constant-order identical pair, compared with a semi-analytic formula
  from the autocorrelation area of a triangle;
* variable s and kappa on vertex-, edge- and identical pairs, compared with a
  brute-force integral in relative coordinates (tests/_bruteforce.py);
* the 1D rules (reading R14) against graded brute force.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from _bruteforce import _bary_grad, _tri_rule, identical_constant_s, pair_reference

P = np.array([[0.1, 0.05], [0.45, 0.12], [0.3, 0.4]])          # tau (stored order)
QV = np.array([[0.1, 0.05], [-0.2, -0.1], [0.05, -0.3]])        # shares P0
QE = np.array([[0.1, 0.05], [0.45, 0.12], [0.35, -0.2]])        # shares P0, P1
CASES = [  # name, type, Q, local dof -> P index, local dof -> Q index
    ("vertex", 1, QV, [0, 1, 2, -1, -1], [0, -1, -1, 1, 2]),
    ("edge", 2, QE, [0, 1, 2, -1], [0, 1, -1, 2]),
    ("identical", 3, P, [0, 1, 2], [0, 1, 2]),
]


def _exact_poly(Pc, Qc, locP, locQ, expo, n=8):
    """int int (psi_i(x)-psi_i(y))(psi_j(x)-psi_j(y)) |x-y|^expo, expo even >= 0,
    by a product of collapsed Gauss rules (exact for these polynomials)."""
    tx, tw = _tri_rule(n)

    def pts(T):
        J = np.stack([T[1] - T[0], T[2] - T[0]], axis=1)
        return T[0] + tx @ J.T, tw * abs(np.linalg.det(J))

    X, WX = pts(Pc)
    Y, WY = pts(Qc)
    GP, cP = _bary_grad(Pc)
    GQ, cQ = _bary_grad(Qc)
    lx, ly = X @ GP.T + cP, Y @ GQ.T + cQ
    R2 = ((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
    Kw = R2 ** (expo // 2) * WX[:, None] * WY[None, :]
    nl = len(locP)
    dif = np.zeros((nl, len(X), len(Y)))
    for i in range(nl):
        if locP[i] >= 0:
            dif[i] += lx[:, locP[i]][:, None]
        if locQ[i] >= 0:
            dif[i] -= ly[:, locQ[i]][None, :]
    return np.einsum("iab,jab,ab->ij", dif, dif, Kw)


def _np_field(f):
    def ev(X):
        v = np.full(len(X), f.c0)
        for r in f.fourier:
            v = v + r[3] * np.cos(math.pi * (X @ r[:2]) + r[4])
        return v
    return ev


def test_gauss_legendre_exactness():
    for n in (1, 2, 3, 5, 9, 16):
        x, w = oracle.gauss01(n)
        for k in range(2 * n):
            assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
        assert np.all(np.diff(x) > 0)


@pytest.mark.parametrize("s,sbar,expo", [(-2.0, 2.0 / 3.0, 2), (-1.0, 0.5, 0)])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_singular_rules_exact_for_polynomial_kernels(case, s, sbar, expo):
    """With s = -2 (gamma = |x-y|^2) and s_bar = 2/3, or s = -1 (gamma = 1) and
    s_bar = 1/2, every factor of the transformed integrands of e:int-v-2,
    e:int-e and e:int-i-2 is a polynomial, so the tensor Gauss rule is exact."""
    name, typ, Q, lp, lq = case
    ref = _exact_poly(P, Q, lp, lq, expo)
    L = oracle.pair_local(2, typ, P, Q, synth.const_field(s), synth.const_field(0.0), sbar, 6)
    assert np.abs(L - ref).max() <= 1e-12 * np.abs(ref).max()


def test_identical_constant_order_semianalytic():
    """Constant s: the identical-pair rule converges to the autocorrelation
    formula (the paper's error law for this pair is algebraic in n because
    of the zeta^((2 sbar - S)/(4 - 2 sbar)) and eta1^(2-S) factors)."""
    s = 0.7
    ref = identical_constant_s(P, s)
    errs = []
    for ns in (3, 6, 12, 24):
        L = oracle.pair_local(2, 3, P, P, synth.const_field(s), synth.const_field(0.0), 0.9, ns)
        errs.append(np.abs(L - ref).max() / np.abs(ref).max())
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 3e-4


def test_vertex_rule_geometric_when_s_equals_sbar():
    """For s = s_bar the zeta exponent vanishes and the vertex-case integrand
    is analytic: the error decays like (2 rho)^(-2n) (Sec. 4.1)."""
    s = 0.45
    c = lambda X: np.full(len(X), s)
    z = lambda X: np.zeros(len(X))
    ref = pair_reference(P, QV, CASES[0][3], CASES[0][4], c, z, n_r=16)
    L = oracle.pair_local(2, 1, P, QV, synth.const_field(s), synth.const_field(0.0), s, 12)
    assert np.abs(L - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_variable_order_against_bruteforce(case):
    """Variable s and kappa: the rule converges to the relative-coordinate
    brute-force integral.  A mistake in how s(x), s(y) or kappa enter (e.g.
    s(x) used for both points) would leave an O(1e-2) gap."""
    name, typ, Q, lp, lq = case
    sF = synth.fourier_field(0.55, [[1, 2, 0, 0.2, 0.3], [2, -1, 0, 0.1, 1.0]])
    kF = synth.fourier_field(0.1, [[1, 1, 0, 0.4, 0.2]])
    ref = pair_reference(P, Q, lp, lq, _np_field(sF), _np_field(kF), n_r=12)
    errs = []
    for ns in (3, 6, 12, 24):
        L = oracle.pair_local(2, typ, P, Q, sF, kF, 0.9, ns)
        errs.append(np.abs(L - ref).max() / np.abs(ref).max())
    assert errs[-1] < 4e-4 and errs[-1] < errs[0] / 8, errs


def _bf_1d(x0, x1, y0, y1, f, levels=40, n=12):
    """int_{x0}^{x1} int_{y0}^{y1} f(x,y) dx dy for two intervals sharing one
    end point, graded towards the shared point in both variables."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1), 0.5 * w

    def graded(a, b, toward):
        # nodes on [a,b] graded towards endpoint `toward`
        L = b - a
        edges = [0.0] + [L * 0.3 ** k for k in range(levels)][::-1]
        xs, ws = [], []
        for i in range(len(edges) - 1):
            e0, e1 = edges[i], edges[i + 1]
            t = e0 + (e1 - e0) * g
            xs.append(t)
            ws.append((e1 - e0) * w)
        t = np.concatenate(xs)
        ww = np.concatenate(ws)
        return (a + t, ww) if toward == a else (b - t, ww)

    shared = x0 if x0 in (y0, y1) else x1
    X, WX = graded(x0, x1, shared)
    Y, WY = graded(y0, y1, shared)
    XX, YY = np.meshgrid(X, Y, indexing="ij")
    return np.sum(WX[:, None] * WY[None, :] * f(XX, YY))


@pytest.mark.parametrize("s", [0.3, 0.6])
def test_1d_rules_against_bruteforce(s):
    """1D identical cell (reading R14) against its closed form, adjacent cells
    against graded brute force; for s = s_bar the adjacent-cell integrand is
    analytic and the rule converges geometrically."""
    h1, h2 = 0.3, 0.2
    # identical cell [0, h1], local [P0, P1]: psi differences are -+z/h1 with
    # z = x - y, so I_ij = 2 g_i g_j int_0^h1 (h1 - z) z^(1-2s) dz in closed form
    gg = np.array([-1.0 / h1, 1.0 / h1])
    val = 2.0 * (h1 * h1 ** (2 - 2 * s) / (2 - 2 * s) - h1 ** (3 - 2 * s) / (3 - 2 * s))
    ref = val * np.outer(gg, gg)
    Pc = np.array([[0.0], [h1]])
    errs = [np.abs(oracle.pair_local(1, 3, Pc, Pc, synth.const_field(s), synth.const_field(0.0), sb, 16)
                   - ref).max() / np.abs(ref).max() for sb in (s, 0.9)]
    # s_bar = 0.9: z = zeta^5 and the zeta-integrand zeta^((1.8-2s)/0.2)(1-zeta^5)
    # is a polynomial for s = 0.3, 0.6, so the rule is exact; s_bar = s leaves
    # (1 - zeta^(1/(2-2s))), integrated to the algebraic rate
    assert errs[1] < 1e-13, errs
    assert errs[0] < 1e-4, errs
    # adjacent cells tau=[0,h1] (stored 0 -> h1) and tau'=[-h2,0] sharing 0
    Pc = np.array([[0.0], [h1]])
    Qc = np.array([[0.0], [-h2]])
    hat = [lambda x, y: (1 - x / h1) - (1 + y / h2),      # shared vertex 0
           lambda x, y: x / h1,                             # tau's other vertex
           lambda x, y: -(-y / h2)]                         # tau''s other vertex
    ref = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            f = lambda x, y, i=i, j=j: hat[i](x, y) * hat[j](x, y) * np.abs(x - y) ** (-1 - 2 * s)
            ref[i, j] = _bf_1d(0.0, h1, -h2, 0.0, f)
    L = oracle.pair_local(1, 1, Pc, Qc, synth.const_field(s), synth.const_field(0.0), s, 12)
    assert np.abs(L - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("s,sbar,expo", [(-1.5, 0.5, 2), (-0.5, 0.5, 0)])
def test_1d_rules_exact_for_polynomial_kernels(s, sbar, expo):
    h1, h2 = 0.3, 0.2
    g, w = np.polynomial.legendre.leggauss(8)
    g, w = 0.5 * (g + 1), 0.5 * w
    # identical
    x = h1 * g
    wx = h1 * w
    phi = [1 - x / h1, x / h1]
    ref = np.zeros((2, 2))
    for i in range(2):
        for j in range(2):
            D = (phi[i][:, None] - phi[i][None, :]) * (phi[j][:, None] - phi[j][None, :])
            ref[i, j] = np.sum(wx[:, None] * wx[None, :] * D * np.abs(x[:, None] - x[None, :]) ** expo)
    Pc = np.array([[0.0], [h1]])
    L = oracle.pair_local(1, 3, Pc, Pc, synth.const_field(s), synth.const_field(0.0), sbar, 8)
    assert np.abs(L - ref).max() < 1e-13 * np.abs(ref).max()
    # adjacent
    y = -h2 * g
    wy = h2 * w
    X, Y = np.meshgrid(x, y, indexing="ij")
    Wt = wx[:, None] * wy[None, :]
    dif = [(1 - X / h1) - (1 + Y / h2), X / h1, Y / h2]
    ref = np.array([[np.sum(Wt * dif[i] * dif[j] * np.abs(X - Y) ** expo) for j in range(3)] for i in range(3)])
    Qc = np.array([[0.0], [-h2]])
    L = oracle.pair_local(1, 1, Pc, Qc, synth.const_field(s), synth.const_field(0.0), sbar, 8)
    assert np.abs(L - ref).max() < 1e-13 * np.abs(ref).max()
