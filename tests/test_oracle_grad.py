"""Pins for the oracle's quasiparticle gradient: central finite differences of
the oracle's own Newton root (converged to 1e-13 Ha) with respect to orbital
energies, factor entries and MO coefficients (the forward path only, not
the gradient formulas), on the tiny case."""
import numpy as np
import pytest

import workloads as W
from oracle import ao2mo, cd, eri, grad, qp, sigma2


@pytest.fixture(scope="module")
def c0():
    m = W.config0()
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    r = cd.decompose(pd, 1e-6)
    Lov, Lp = ao2mo.mo_factors(r.L, m.C, m.nocc, m.orbitals)
    return m, r, Lov, Lp


def root(Lq, Lov, eps, nocc, q):
    def f(x):
        s, d = sigma2.sigma2_from_factors(Lq, Lov, eps, nocc, [x])
        return s[0], d[0]
    w, P, it, st = qp.newton_qp(f, eps[q], conv=1e-13, max_iter=100)
    assert st == qp.QP_OK
    return w


@pytest.mark.parametrize("t", [0, 1])
def test_gradient_matches_central_differences(c0, t):
    m, r, Lov, Lp = c0
    q = int(m.orbitals[t])
    w = root(Lp[t], Lov, m.eps, m.nocc, q)
    d_eps, d_Lq, d_Lov, P = grad.qp_gradient(Lp[t], Lov, m.eps, m.nocc, q, w)
    assert 0 < P <= 1
    h = 1e-6
    for k in [0, 2, q, m.nocc, m.nocc + 3, m.nbf - 1]:
        e1, e2 = m.eps.copy(), m.eps.copy()
        e1[k] += h
        e2[k] -= h
        fd = (root(Lp[t], Lov, e1, m.nocc, q) - root(Lp[t], Lov, e2, m.nocc, q)) / (2 * h)
        assert abs(fd - d_eps[k]) <= 1e-6 * max(1.0, abs(d_eps[k]))
    rng = np.random.default_rng(t)
    for _ in range(5):
        r_, K = rng.integers(m.nbf), rng.integers(Lp.shape[2])
        a, b = Lp[t].copy(), Lp[t].copy()
        a[r_, K] += h
        b[r_, K] -= h
        fd = (root(a, Lov, m.eps, m.nocc, q) - root(b, Lov, m.eps, m.nocc, q)) / (2 * h)
        assert abs(fd - d_Lq[r_, K]) <= 1e-6 * max(1.0, abs(d_Lq[r_, K]))
        i, a_ = rng.integers(m.nocc), rng.integers(m.nbf - m.nocc)
        A, B = Lov.copy(), Lov.copy()
        A[i, a_, K] += h
        B[i, a_, K] -= h
        fd = (root(Lp[t], A, m.eps, m.nocc, q) - root(Lp[t], B, m.eps, m.nocc, q)) / (2 * h)
        assert abs(fd - d_Lov[i, a_, K]) <= 1e-6 * max(1.0, abs(d_Lov[i, a_, K]))


def test_coefficient_gradient_matches_central_differences(c0):
    m, r, Lov, Lp = c0
    t = 1
    q = int(m.orbitals[t])
    w = root(Lp[t], Lov, m.eps, m.nocc, q)
    d_eps, d_Lq, d_Lov, P = grad.qp_gradient(Lp[t], Lov, m.eps, m.nocc, q, w)
    d_Lp = np.zeros_like(Lp)
    d_Lp[t] = d_Lq
    dC = grad.transform_gradient(r.L, m.C, m.nocc, m.orbitals, d_Lov, d_Lp)
    h = 1e-6
    rng = np.random.default_rng(5)
    for _ in range(6):
        mu, p = rng.integers(m.nbf), rng.integers(m.nbf)
        C1, C2 = m.C.copy(), m.C.copy()
        C1[mu, p] += h
        C2[mu, p] -= h
        vals = []
        for Cx in (C1, C2):
            lov, lp = ao2mo.mo_factors(r.L, Cx, m.nocc, m.orbitals)
            vals.append(root(lp[t], lov, m.eps, m.nocc, q))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dC[mu, p]) <= 1e-6 * max(1.0, abs(dC[mu, p]))
