"""Pins for the oracle's integrals (Sec. II.A, Eq. integral), independent of its formula.

* Boys F0 against adaptive quadrature of int_0^1 exp(-T u^2) du.
* The Gaussian product theorem: chi_mu * chi_nu evaluated point by point.
* The Coulomb energy of two spherical Gaussian clouds by the shell theorem
  (enclosed charge by Gauss-Legendre quadrature, no erf), which with the
  product theorem fixes every four-centre s-type ERI.
* Textbook limits: self-repulsion 2 sqrt(a/pi) of a normalised s-Gaussian
  density, and 1/R for distant clouds.
* Symmetry and positive semi-definiteness of the supermatrix.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy.integrate import quad

import workloads as W
from oracle import eri


def _gl(a, b, n):
    x, w = leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def cloud_coulomb(p, q, R, n=200, nq=80):
    """Coulomb energy of unit Gaussian clouds (exponents p at 0, q at distance R)
    by direct quadrature: potential of the q-cloud from the shell theorem."""
    def rho(e, r):
        return (e / math.pi) ** 1.5 * np.exp(-e * r * r)
    r, wr = _gl(0.0, 9.0 / math.sqrt(p), n)
    mu, wm = _gl(-1.0, 1.0, n)
    s = np.sqrt(np.maximum(r[:, None] ** 2 + R * R - 2 * r[:, None] * R * mu[None, :], 0.0))
    t, wt = leggauss(nq)
    tt = 0.5 * s[..., None] * (t + 1.0)
    ww = 0.5 * s[..., None] * wt
    enclosed = (4 * math.pi * tt ** 2 * rho(q, tt) * ww).sum(-1)
    outer = 4 * math.pi * (q / math.pi) ** 1.5 * np.exp(-q * s * s) / (2 * q)
    phi = np.where(s > 0, enclosed / np.where(s > 0, s, 1.0), 0.0) + outer
    return float((2 * math.pi * wr[:, None] * wm[None, :] * r[:, None] ** 2
                  * rho(p, r)[:, None] * phi).sum())


@pytest.mark.parametrize("T", [0.0, 1e-14, 1e-9, 1e-6, 1e-3, 0.1, 1.0, 7.5, 30.0, 300.0, 5e3])
def test_boys_f0_matches_quadrature(T):
    ref, _ = quad(lambda u: math.exp(-T * u * u), 0.0, 1.0, epsabs=1e-17, epsrel=1e-13, limit=200)
    assert abs(float(eri.boys_f0(T)) - ref) <= 2e-15 * max(ref, 1e-300) + 1e-17


def test_gaussian_product_theorem():
    rng = np.random.default_rng(11)
    xyz = rng.uniform(-2, 2, size=(5, 3))
    alpha = rng.uniform(0.1, 8.0, size=5)
    pd = eri.PairData(xyz, alpha)
    pts = rng.uniform(-3, 3, size=(50, 3))
    norm = (2 * alpha / math.pi) ** 0.75
    for I in range(pd.npair):
        m, n = pd.mu[I], pd.nu[I]
        direct = (norm[m] * np.exp(-alpha[m] * ((pts - xyz[m]) ** 2).sum(1))
                  * norm[n] * np.exp(-alpha[n] * ((pts - xyz[n]) ** 2).sum(1)))
        prod = pd.K[I] * np.exp(-pd.p[I] * ((pts - pd.P[I]) ** 2).sum(1))
        np.testing.assert_allclose(prod, direct, rtol=1e-12, atol=1e-300)


def test_four_centre_eri_against_shell_theorem_quadrature():
    rng = np.random.default_rng(5)
    xyz = rng.uniform(-1.5, 1.5, size=(4, 3))
    alpha = np.array([0.3, 1.7, 0.9, 6.0])
    pd = eri.PairData(xyz, alpha)
    for I, J in [(eri.pair_index(0, 1), eri.pair_index(2, 3)),
                 (eri.pair_index(0, 0), eri.pair_index(3, 3)),
                 (eri.pair_index(1, 2), eri.pair_index(1, 2)),
                 (eri.pair_index(0, 3), eri.pair_index(1, 1))]:
        p, q = pd.p[I], pd.p[J]
        R = float(np.linalg.norm(pd.P[I] - pd.P[J]))
        charge = pd.K[I] * (math.pi / p) ** 1.5 * pd.K[J] * (math.pi / q) ** 1.5
        ref = charge * cloud_coulomb(p, q, R)
        got = float(eri.eri_from_pairs(pd, np.array([I]), np.array([J]))[0])
        assert abs(got - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("a", [0.08, 0.5, 2.0, 30.0])
def test_self_repulsion_closed_form(a):
    pd = eri.PairData(np.zeros((1, 3)), np.array([a]))
    assert abs(eri.eri_diagonal(pd)[0] - 2.0 * math.sqrt(a / math.pi)) < 1e-14 * a ** 0.5


def test_point_charge_limit():
    R = 60.0
    pd = eri.PairData(np.array([[0.0, 0, 0], [R, 0, 0]]), np.array([5.0, 7.0]))
    v = eri.eri_from_pairs(pd, np.array([eri.pair_index(0, 0)]), np.array([eri.pair_index(1, 1)]))[0]
    assert abs(v - 1.0 / R) < 1e-15


def test_supermatrix_symmetric_psd_and_eightfold():
    m = W.config0()
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    V = eri.eri_matrix(pd)
    assert np.array_equal(V, V.T) or np.abs(V - V.T).max() < 1e-15
    w = np.linalg.eigvalsh(V)
    assert w.min() > -1e-12 * w.max()
    g = eri.eri_tensor(pd)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        np.testing.assert_allclose(g, g.transpose(perm), rtol=0, atol=1e-15)
    # Schwarz: |V_IJ| <= sqrt(V_II V_JJ) (far pairs underflow to ~1e-170 or 0)
    assert np.all(np.abs(V) <= np.sqrt(np.outer(np.diag(V), np.diag(V))) * (1 + 1e-12) + 1e-150)
