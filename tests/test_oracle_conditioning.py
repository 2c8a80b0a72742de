"""Pin P9: the condition number of the assembled stiffness matrix grows like
h^(-2s) under refinement (Sec. 7: the CG condition estimate is about
O(h^(-2 s*)); for a quasi-uniform mesh lambda_max ~ h^(d-2s) and lambda_min ~
h^d).  Eigenvalues of the oracle's A = B + K + M by a dense symmetric solver.

* 1D, constant s = 0.3, a = C_{1,s}/2, exterior tail: halving h multiplies
  kappa(A) by 2^(2s) (log2 ratio 0.6);
* 2D disk, constant s = 0.7, kappa = 1, bounded annular exterior: the log2
  ratio per halving of h approaches 2s = 1.4.
"""
import math

import numpy as np

import oracle
import synth


def _kappa(ref):
    ev = np.linalg.eigvalsh(ref.B + ref.K + ref.M)
    assert ev[0] > 0
    return ev[-1] / ev[0]


def test_condition_growth_1d():
    s = 0.3
    a = synth.const_field(math.log(synth.frac_laplacian_const(1, s) / 2))
    kap = []
    for n in (32, 64, 128, 256):
        m = synth.interval_mesh(n, R=1.1)
        kap.append(_kappa(oracle.assemble(m, synth.const_field(s), a, s_bar=0.3, n_sing=3, tail=1, R=1.1)))
    rates = [math.log(b / c, 2) for c, b in zip(kap, kap[1:])]
    assert all(abs(r - 2 * s) < 0.03 for r in rates), rates


def test_condition_growth_2d():
    s = 0.7
    kap = []
    for K in (6, 12, 24):
        m = synth.disk_mesh(K, R=1.1, jitter=0.2, seed=K)
        kap.append(_kappa(oracle.assemble(m, synth.const_field(s), synth.const_field(0.0), s_bar=0.9, n_sing=3)))
    rates = [math.log(b / c, 2) for c, b in zip(kap, kap[1:])]
    assert 1.0 < rates[0] < 1.8 and abs(rates[-1] - 2 * s) < 0.25, rates
