"""Pins for the oracle's transform, self-energy and Newton solve.

* Eq. transformation + Eq. aomo at delta = 0 equal the conventional O(N^5)
  four-index transform of the explicit AO integrals; C = 1 is unpacking.
* Eq. SE from factors equals (a) the explicit-MO-integral sum, (b) an
  independent spin-orbital derivation with antisymmetrised integrals and
  explicit spin sums, (c) the MP2 identity sum_i Sigma^(2p1h)_ii(e_i) = E_MP2
  = -sum_a Sigma^(2h1p)_aa(e_a) with E_MP2 from Eq. MP2, and (d) the
  one-occupied/one-virtual closed form.
* Eq. MP2 from the factors equals the explicit-integral loop, splits per
  occupied orbital into the 2p1h self-energy at e_i, and reduces to the
  o = v = 1 closed form.
* dSigma/dw equals a central difference; every pole residue is >= 0, so
  dSigma/dw < 0 and 0 < P <= 1 (Eq. ps).
* Newton (Eq. iter) converges to a root of w = e_q + Sigma(w) that a
  bracketing solver confirms inside the pole-free interval.
"""
import numpy as np
import pytest
from scipy.optimize import brentq

import workloads as W
from oracle import ao2mo, cd, eri, qp, sigma2


@pytest.fixture(scope="module")
def c0():
    m = W.config0()
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    r = cd.decompose(pd, 0.0)
    g4 = ao2mo.ao_to_mo_4index(eri.eri_tensor(pd), m.C)
    Lov, Lp = ao2mo.mo_factors(r.L, m.C, m.nocc, np.arange(m.nbf))
    return m, pd, r, g4, Lov, Lp


def test_factor_transform_matches_four_index(c0):
    m, pd, r, g4, Lov, Lp = c0
    g = ao2mo.mo_integrals(ao2mo.transform_full(r.L, m.C))
    assert np.abs(g - g4).max() <= 1e-11 * np.abs(g4).max()


def test_identity_coefficients_unpack():
    m = W.config0()
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    r = cd.decompose(pd, 1e-6)
    B = ao2mo.transform_full(r.L, np.eye(m.nbf))
    for K in (0, r.M // 2, r.M - 1):
        for I in range(0, pd.npair, 7):
            assert B[K, pd.mu[I], pd.nu[I]] == r.L[K, I] == B[K, pd.nu[I], pd.mu[I]]


def test_blocks_match_full_transform(c0):
    m, pd, r, g4, Lov, Lp = c0
    B = ao2mo.transform_full(r.L, m.C)
    np.testing.assert_allclose(Lov, B[:, :m.nocc, m.nocc:].transpose(1, 2, 0), atol=1e-13)
    np.testing.assert_allclose(Lp, B.transpose(1, 2, 0), atol=1e-13)


@pytest.mark.parametrize("q", [0, 3, 5, 6, 11, 23])
def test_sigma_factors_vs_mo_integrals_and_spin_orbital(c0, q):
    m, pd, r, g4, Lov, Lp = c0
    E = W.energy_grid(m.eps[[q]], 3, 0.1)[0]
    s, ds = sigma2.sigma2_from_factors(Lp[q], Lov, m.eps, m.nocc, E)
    s_mo = sigma2.sigma2_from_mo_integrals(g4, m.eps, m.nocc, q, E)
    np.testing.assert_allclose(s, s_mo, rtol=1e-11, atol=1e-12)
    for k in range(len(E)):
        s_so = sigma2.sigma2_spin_orbital(g4, m.eps, m.nocc, q, E[k])
        assert abs(s[k] - s_so) <= 1e-11 * max(1.0, abs(s_so))


def test_mp2_identity(c0):
    m, pd, r, g4, Lov, Lp = c0
    emp2 = sigma2.mp2_energy(g4, m.eps, m.nocc)
    occ_sum = sum(sigma2.sigma2_from_factors(Lp[i], Lov, m.eps, m.nocc, [m.eps[i]], parts=True)[1][0]
                  for i in range(m.nocc))
    vir_sum = sum(sigma2.sigma2_from_factors(Lp[a], Lov, m.eps, m.nocc, [m.eps[a]], parts=True)[0][0]
                  for a in range(m.nocc, m.nbf))
    assert emp2 < 0
    assert abs(occ_sum - emp2) <= 1e-12 * abs(emp2)
    assert abs(vir_sum + emp2) <= 1e-12 * abs(emp2)


def test_mp2_from_factors_pins(c0):
    """Eq. MP2 from the factors against the explicit-integral quadruple loop
    (an O(N^5) transform of the explicit AO tensor, delta = 0), the per-i
    split against the 2p1h self-energy at e_i, and the o = v = 1 closed form
    (ia|ia)^2 / (2 (e_i - e_a))."""
    m, pd, r, g4, Lov, Lp = c0
    e_fac = sigma2.mp2_from_factors(Lov, m.eps, m.nocc)
    assert abs(e_fac - sigma2.mp2_energy(g4, m.eps, m.nocc)) <= 1e-11 * abs(e_fac)
    e_i = sigma2.mp2_from_factors(Lov, m.eps, m.nocc, pairs=True)
    for i in range(m.nocc):
        two_p1h = sigma2.sigma2_from_factors(Lp[i], Lov, m.eps, m.nocc, [m.eps[i]], parts=True)[1][0]
        assert abs(e_i[i] - two_p1h) <= 1e-12 * abs(e_fac)
    assert np.all(e_i < 0)
    rng = np.random.default_rng(5)
    L1 = rng.standard_normal((1, 1, 7))
    eps = np.array([-0.6, 0.4])
    x = float(L1[0, 0] @ L1[0, 0])
    assert sigma2.mp2_from_factors(L1, eps, 1) == pytest.approx(x * x / (2 * (-0.6 - 0.4)), rel=1e-14)


def test_one_occupied_one_virtual_closed_form():
    rng = np.random.default_rng(3)
    M = 5
    Lq = rng.standard_normal((2, M))          # rows: occupied i, virtual a
    Lov = rng.standard_normal((1, 1, M))
    eps = np.array([-0.7, 0.4])
    w = -0.2
    qi, qa = Lq[0] @ Lov[0, 0], Lq[1] @ Lov[0, 0]    # (qi|ai), (qa|ia)
    closed = qi ** 2 / (w + eps[1] - 2 * eps[0]) + qa ** 2 / (w + eps[0] - 2 * eps[1])
    s, _ = sigma2.sigma2_from_factors(Lq, Lov, eps, 1, [w])
    assert abs(s[0] - closed) <= 1e-14 * abs(closed)


def test_derivative_central_difference_and_sign(c0):
    m, pd, r, g4, Lov, Lp = c0
    for q in (5, 6):
        E = W.energy_grid(m.eps[[q]], 5, 0.05)[0]
        s, ds = sigma2.sigma2_from_factors(Lp[q], Lov, m.eps, m.nocc, E)
        h = 1e-5
        sp, _ = sigma2.sigma2_from_factors(Lp[q], Lov, m.eps, m.nocc, E + h)
        sm, _ = sigma2.sigma2_from_factors(Lp[q], Lov, m.eps, m.nocc, E - h)
        np.testing.assert_allclose(ds, (sp - sm) / (2 * h), rtol=1e-7)
        assert np.all(ds < 0)


def test_pole_residues_nonnegative(c0):
    """Pair (a,b) and (b,a) share a denominator; their summed numerator
    2x^2 + 2y^2 - 2xy is >= 0, so Sigma has positive residues."""
    m, pd, r, g4, Lov, Lp = c0
    q = 6
    U = np.einsum("ak,ibk->aib", Lp[q][m.nocc:], Lov)
    pair = (2 * U - U.transpose(2, 1, 0)) * U
    assert np.all(pair + pair.transpose(2, 1, 0) >= -1e-15)


@pytest.mark.parametrize("q", [5, 6])
def test_newton_root_confirmed_by_bracketing(c0, q):
    m, pd, r, g4, Lov, Lp = c0

    def f(w):
        s, ds = sigma2.sigma2_from_factors(Lp[q], Lov, m.eps, m.nocc, [w])
        return s[0], ds[0]
    w, P, it, st = qp.newton_qp(f, m.eps[q], conv=1e-12)
    assert st == qp.QP_OK and 0 < P <= 1
    assert abs(w - m.eps[q] - f(w)[0]) < 1e-11
    # pole-free interval around the root: nearest poles of either sum
    eo, ev = m.eps[:m.nocc], m.eps[m.nocc:]
    poles = np.concatenate([(eo[:, None, None] + eo[None, None, :] - ev[None, :, None]).ravel(),
                            (ev[:, None, None] + ev[None, None, :] - eo[None, :, None]).ravel()])
    lo = poles[poles < w].max() + 1e-9
    hi = poles[poles > w].min() - 1e-9
    root = brentq(lambda x: x - m.eps[q] - f(x)[0], lo, hi, xtol=1e-14)
    assert abs(root - w) < 1e-10


def test_newton_reports_non_convergence(c0):
    m, pd, r, g4, Lov, Lp = c0

    def f(w):
        s, ds = sigma2.sigma2_from_factors(Lp[5], Lov, m.eps, m.nocc, [w])
        return s[0], ds[0]
    w, P, it, st = qp.newton_qp(f, m.eps[5], conv=1e-5, max_iter=1)
    assert st == qp.QP_NO_CONVERGENCE and it == 1


def test_bracketed_qp_finds_the_unique_root_of_the_pole_free_interval(c0):
    """Safeguarded Newton: its root is the one brentq finds between the two
    poles nearest e_q (an independent bracketing solver), with 0 < P <= 1;
    where plain Newton stays in that interval it finds the same root; the
    bracket comes from a direct loop over the Eq. SE denominators."""
    m, pd, r, g4, Lov, Lp = c0
    found = 0
    for q in range(m.nbf):
        def f(x, q=q):
            a, d = sigma2.sigma2_from_factors(Lp[q], Lov, m.eps, m.nocc, [x])
            return a[0], d[0]
        lo, hi = qp.pole_bracket(m.eps, m.nocc, m.eps[q])
        # the bracket by a plain loop over every denominator
        o = m.nocc
        den = [m.eps[i] + m.eps[j] - m.eps[a] for i in range(o) for j in range(o)
               for a in range(o, m.nbf)]
        den += [m.eps[a] + m.eps[b] - m.eps[i] for a in range(o, m.nbf) for b in range(o, m.nbf)
                for i in range(o)]
        den = np.array(den)
        assert lo == den[den < m.eps[q]].max() and hi == den[den > m.eps[q]].min()
        w, P, it, st = qp.bracketed_qp(f, m.eps[q], lo, hi, conv=1e-12, max_iter=200)
        assert st == qp.QP_OK and lo < w < hi and 0 < P <= 1
        root = brentq(lambda x: x - m.eps[q] - f(x)[0], lo + 1e-12 * abs(lo), hi - 1e-12 * abs(hi),
                      xtol=1e-14)
        assert abs(w - root) <= 1e-10
        wn, Pn, itn, stn = qp.newton_qp(f, m.eps[q], conv=1e-12, max_iter=200)
        if stn == qp.QP_OK and lo < wn < hi:
            assert abs(wn - w) <= 1e-10
            found += 1
    assert found >= 1
