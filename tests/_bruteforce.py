"""Independent reference integrals for touching element pairs.

These do not use the paper's Duffy-type maps.  They integrate

    I_ij = int_tau int_tau' a(x,y) (psi_i(x)-psi_i(y)) (psi_j(x)-psi_j(y)) / |x-y|^(d+s(x)+s(y))

in relative coordinates z = x - y = r e(theta):

    I = int_theta int_r r int_{y in tau' ∩ (tau - z)} F(y+z, y) dy dr dtheta,

clipping the two triangles for every (theta, r), splitting r at every
vertex/edge crossing of the two triangles, grading r geometrically towards 0
and splitting theta at every direction where an edge of either triangle is
parallel to e.  With constant s and the identical pair the inner area has a
closed form, giving a one-dimensional semi-analytic reference.
"""
from __future__ import annotations

import math

import numpy as np


def gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _bary_grad(P):
    """Affine barycentric coordinates of triangle P (3x2): lam(y) = G y + c."""
    A = np.array([[P[0, 0], P[1, 0], P[2, 0]], [P[0, 1], P[1, 1], P[2, 1]], [1.0, 1.0, 1.0]])
    Ai = np.linalg.inv(A)            # lam = Ai @ [y;1]
    return Ai[:, :2], Ai[:, 2]


def _clip(poly, G, c, shift):
    """Clip polygon (list of 2-vectors) by half-planes G y + c + G shift >= 0."""
    out = poly
    for k in range(3):
        g, cc = G[k], c[k] + G[k] @ shift
        if not out:
            return out
        new = []
        n = len(out)
        for i in range(n):
            p, q = out[i], out[(i + 1) % n]
            fp, fq = g @ p + cc, g @ q + cc
            if fp >= 0:
                new.append(p)
            if (fp >= 0) != (fq >= 0):
                t = fp / (fp - fq)
                new.append(p + t * (q - p))
        out = new
    return out


_TX, _TW = None, None


def _tri_rule(n=6):
    """Collapsed Gauss rule on the unit simplex (0,0),(1,0),(0,1)."""
    x, w = gauss01(n)
    U, V = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    a = U.ravel()
    b = (V * (1 - U)).ravel()
    ww = (WU * WV * (1 - U)).ravel()
    return np.stack([a, b], axis=1), ww


def pair_reference(P, Q, loc_is_P, loc_is_Q, sfun, kfun, n_theta=12, n_r=10, levels=18, n_tri=6):
    """Brute-force local matrix for triangles P, Q (3x2 each).

    loc_is_P[a] = index (0..2) of the local DoF a in P or -1; same for Q.
    sfun(X) and kfun(X) evaluate s and log kappa at points X (n,2).
    """
    P = np.asarray(P, float)
    Q = np.asarray(Q, float)
    nl = len(loc_is_P)
    GP, cP = _bary_grad(P)
    GQ, cQ = _bary_grad(Q)
    tx, tw = _tri_rule(n_tri)
    # theta breakpoints: normals of all edges (directions where an edge is
    # parallel to e) and directions of the vertex differences
    brk = []
    for G in (GP, GQ):
        for k in range(3):
            ang = math.atan2(G[k, 1], G[k, 0])
            brk += [ang + math.pi / 2, ang - math.pi / 2]
    for a in range(3):
        for b in range(3):
            dz = P[a] - Q[b]
            if np.linalg.norm(dz) > 1e-14:
                brk.append(math.atan2(dz[1], dz[0]))
    brk = sorted({(x % (2 * math.pi)) for x in brk})
    brk = brk + [brk[0] + 2 * math.pi]
    gth, wth = gauss01(n_theta)
    gr, wr = gauss01(n_r)
    diffs = np.array([P[a] - Q[b] for a in range(3) for b in range(3)])
    # half-planes n.z <= h of the support set conv{P_a - Q_b} of z = x - y
    from scipy.spatial import ConvexHull
    eq = ConvexHull(diffs).equations
    I = np.zeros((nl, nl))
    for it in range(len(brk) - 1):
        t0, t1 = brk[it], brk[it + 1]
        if t1 - t0 < 1e-14:
            continue
        for th, wt in zip(t0 + (t1 - t0) * gth, (t1 - t0) * wth):
            e = np.array([math.cos(th), math.sin(th)])
            # r_max: exit distance of the ray r e from the support set of z
            ne = eq[:, :2] @ e
            pos = ne > 1e-14
            rmax = float(np.min(-eq[pos, 2] / ne[pos])) if np.any(pos) else 0.0
            if rmax <= 1e-14:
                continue
            # r breakpoints: vertex of (tau - r e) on an edge line of tau', and
            # vertex of tau' on an edge line of (tau - r e)
            rb = [0.0, rmax]
            for a in range(3):
                for k in range(3):
                    den = GQ[k] @ e
                    if abs(den) > 1e-14:
                        r = (GQ[k] @ P[a] + cQ[k]) / den
                        if 0 < r < rmax:
                            rb.append(r)
                    den = GP[k] @ e
                    if abs(den) > 1e-14:
                        r = -(GP[k] @ Q[a] + cP[k]) / den
                        if 0 < r < rmax:
                            rb.append(r)
            # drop round-off events at r ~ 0 so the graded first interval
            # really starts at the singular point r = 0
            rb = sorted({r for r in rb if r == 0.0 or r > 1e-9 * rmax})
            rs, wrs = [], []
            for j in range(len(rb) - 1):
                a0, a1 = rb[j], rb[j + 1]
                if j == 0:
                    # geometric grading towards r = 0
                    edges = [a1 * 0.2 ** l for l in range(levels)][::-1]
                    edges = [0.0] + edges
                    for l in range(len(edges) - 1):
                        b0, b1 = edges[l], edges[l + 1]
                        rs += list(b0 + (b1 - b0) * gr)
                        wrs += list((b1 - b0) * wr)
                else:
                    rs += list(a0 + (a1 - a0) * gr)
                    wrs += list((a1 - a0) * wr)
            for r, wrr in zip(rs, wrs):
                z = r * e
                poly = _clip([Q[0].copy(), Q[1].copy(), Q[2].copy()], GP, cP, z)
                if len(poly) < 3:
                    continue
                Ys, Ws = [], []
                p0 = poly[0]
                for m in range(1, len(poly) - 1):
                    p1, p2 = poly[m], poly[m + 1]
                    J = np.stack([p1 - p0, p2 - p0], axis=1)
                    area2 = abs(np.linalg.det(J))
                    Ys.append(p0 + tx @ J.T)
                    Ws.append(tw * area2)
                Y = np.concatenate(Ys)
                W = np.concatenate(Ws)
                X = Y + z
                lx = X @ GP.T + cP           # barycentric of x in P
                ly = Y @ GQ.T + cQ           # barycentric of y in Q
                S = sfun(X) + sfun(Y)
                aa = np.exp(0.5 * (kfun(X) + kfun(Y)))
                base = W * aa * r ** (-(2.0 + S)) * r * wrr * wt
                dif = np.zeros((nl, len(W)))
                for i in range(nl):
                    if loc_is_P[i] >= 0:
                        dif[i] += lx[:, loc_is_P[i]]
                    if loc_is_Q[i] >= 0:
                        dif[i] -= ly[:, loc_is_Q[i]]
                I += (dif * base) @ dif.T
    return I


def identical_constant_s(P, s, a=1.0, n=40):
    """Semi-analytic identical-pair local matrix for constant s and a:
    I_ij = a |T| B(2-2s, 3) int_0^{2pi} (g_i.e)(g_j.e) m(theta)^(2s-2) dtheta,
    m = sum_k max(0, grad lam_k . e), from the autocorrelation area
    |T ∩ (T+z)| = |T| (1 - sum_k max(0, grad lam_k . z))^2."""
    P = np.asarray(P, float)
    G, _ = _bary_grad(P)
    area = 0.5 * abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0]], axis=1)))
    beta = math.gamma(2 - 2 * s) * math.gamma(3) / math.gamma(5 - 2 * s)
    brk = []
    for k in range(3):
        ang = math.atan2(G[k, 1], G[k, 0])
        brk += [(ang + math.pi / 2) % (2 * math.pi), (ang - math.pi / 2) % (2 * math.pi)]
    brk = sorted(set(brk))
    brk = brk + [brk[0] + 2 * math.pi]
    x, w = gauss01(n)
    I = np.zeros((3, 3))
    for i in range(len(brk) - 1):
        t0, t1 = brk[i], brk[i + 1]
        th = t0 + (t1 - t0) * x
        wt = (t1 - t0) * w
        E = np.stack([np.cos(th), np.sin(th)], axis=1)
        ge = E @ G.T                     # (n, 3): grad lam_k . e
        m = np.sum(np.maximum(ge, 0.0), axis=1)
        f = wt * m ** (2 * s - 2)
        I += (ge * f[:, None]).T @ ge
    return a * area * beta * I
