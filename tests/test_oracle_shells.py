"""Pins of the contracted-shell integrals (oracle/shells.py) by facts fixed
outside its own formulas:

* Boys F_n(T) against adaptive quadrature of int_0^1 u^2n exp(-T u^2) du;
* s-type one-primitive functions give the pinned closed-form s-integrals of
  oracle/eri.py (Eq. integral);
* a p (d) primitive is a centre derivative of an s primitive:
  x_A exp(-a|r-A|^2) = (1/2a) d/dA_x exp(-a|r-A|^2),
  x_A^2 exp(...) = (1/4a^2) d^2/dA_x^2 exp(...) + (1/2a) exp(...),
  x_A y_A exp(...) = (1/4a^2) d^2/(dA_x dA_y) exp(...),
  so central differences of the s-integrals with respect to the centres pin
  every p and d slot (bra and ket);
* 8-fold permutational symmetry, a positive semidefinite supermatrix and the
  Schwarz inequality on a small s/p/d basis;
* every generated function has unit self-overlap (overlap by the same
  Hermite expansion, pinned for s by the closed form exp(-ab/p R^2) (pi/p)^1.5).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

import workloads as W
from oracle import eri as E
from oracle import shells as S


def test_boys_against_quadrature():
    for n in range(9):
        for T in (0.0, 1e-9, 0.3, 2.5, 11.0, 27.0, 60.0):
            ref = quad(lambda u: u ** (2 * n) * math.exp(-T * u * u), 0.0, 1.0, epsabs=0,
                       epsrel=1e-13, limit=200)[0]
            assert abs(float(S.boys(n, T)) - ref) <= 1e-12 * max(ref, 1e-300) + 1e-16, (n, T)


def s_unnormalised(A, a, B, b, C, c, D, d):
    """[ss|ss] over unnormalised s primitives from the pinned closed form."""
    pd = E.PairData(np.array([A, B, C, D], float), np.array([a, b, c, d], float))
    nrm = [(2 * x / math.pi) ** 0.75 for x in (a, b, c, d)]
    I = E.pair_index(0, 1)
    J = E.pair_index(2, 3)
    return float(E.eri_from_pairs(pd, np.array([I]), np.array([J]))[0]) / np.prod(nrm)


def test_s_functions_reduce_to_closed_form():
    rng = np.random.default_rng(0)
    xyz = rng.uniform(0, 3, (4, 3))
    al = np.array([0.3, 1.7, 0.8, 5.0])
    sb = S.ShellBasis(xyz, np.zeros((4, 3), int), np.arange(5), al,
                      (2 * al / math.pi) ** 0.75, np.arange(4))
    sp = S.ShellPairs(sb)
    pd = E.PairData(xyz, al)
    for J in range(pd.npair):
        np.testing.assert_allclose(sp.column(J), E.eri_column(pd, J), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("slot", [0, 1, 2, 3])
def test_p_and_d_are_centre_derivatives_of_s(slot):
    rng = np.random.default_rng(1 + slot)
    cen = rng.uniform(0, 2.5, (4, 3))
    ex = rng.uniform(0.4, 2.0, 4)
    h = 1e-4

    def s_val(c):
        return s_unnormalised(c[0], ex[0], c[1], ex[1], c[2], ex[2], c[3], ex[3])

    def shifted(ax, step, ax2=None, step2=0.0):
        c = cen.copy()
        c[slot, ax] += step
        if ax2 is not None:
            c[slot, ax2] += step2
        return c

    a = ex[slot]
    for ax in range(3):
        # p slot
        lm = [(0, 0, 0)] * 4
        comp = [0, 0, 0]
        comp[ax] = 1
        lm[slot] = tuple(comp)
        val = S.primitive_eri(ex[0], cen[0], lm[0], ex[1], cen[1], lm[1], ex[2], cen[2], lm[2],
                              ex[3], cen[3], lm[3])
        fd = (s_val(shifted(ax, h)) - s_val(shifted(ax, -h))) / (2 * h) / (2 * a)
        assert abs(val - fd) <= 2e-8 * max(abs(fd), 1e-3), ("p", ax, val, fd)
        # d slot, diagonal component x_A^2
        comp = [0, 0, 0]
        comp[ax] = 2
        lm[slot] = tuple(comp)
        val = S.primitive_eri(ex[0], cen[0], lm[0], ex[1], cen[1], lm[1], ex[2], cen[2], lm[2],
                              ex[3], cen[3], lm[3])
        hd = 1e-3
        d2 = (s_val(shifted(ax, hd)) - 2 * s_val(cen) + s_val(shifted(ax, -hd))) / hd ** 2
        fd = d2 / (4 * a * a) + s_val(cen) / (2 * a)
        assert abs(val - fd) <= 2e-6 * max(abs(fd), 1e-3), ("dxx", ax, val, fd)
    # d slot, off-diagonal component x_A y_A
    for ax, ax2 in ((0, 1), (0, 2), (1, 2)):
        comp = [0, 0, 0]
        comp[ax] = 1
        comp[ax2] = 1
        lm = [(0, 0, 0)] * 4
        lm[slot] = tuple(comp)
        val = S.primitive_eri(ex[0], cen[0], lm[0], ex[1], cen[1], lm[1], ex[2], cen[2], lm[2],
                              ex[3], cen[3], lm[3])
        hd = 1e-3
        mixed = (s_val(shifted(ax, hd, ax2, hd)) - s_val(shifted(ax, hd, ax2, -hd))
                 - s_val(shifted(ax, -hd, ax2, hd)) + s_val(shifted(ax, -hd, ax2, -hd))) / (4 * hd * hd)
        fd = mixed / (4 * a * a)
        assert abs(val - fd) <= 2e-6 * max(abs(fd), 1e-3), ("dxy", ax, ax2, val, fd)


def test_p_on_two_centres_is_a_mixed_derivative():
    """(p_x s|p_z s) = (1/2a)(1/2c) d^2/(dA_x dC_z) [ss|ss]."""
    rng = np.random.default_rng(9)
    cen = rng.uniform(0, 2.5, (4, 3))
    ex = rng.uniform(0.4, 2.0, 4)
    lm = [(1, 0, 0), (0, 0, 0), (0, 0, 1), (0, 0, 0)]
    val = S.primitive_eri(ex[0], cen[0], lm[0], ex[1], cen[1], lm[1], ex[2], cen[2], lm[2],
                          ex[3], cen[3], lm[3])
    h = 1e-3

    def sv(dx, dz):
        c = cen.copy()
        c[0, 0] += dx
        c[2, 2] += dz
        return s_unnormalised(c[0], ex[0], c[1], ex[1], c[2], ex[2], c[3], ex[3])
    mixed = (sv(h, h) - sv(h, -h) - sv(-h, h) + sv(-h, -h)) / (4 * h * h)
    fd = mixed / (4 * ex[0] * ex[2])
    assert abs(val - fd) <= 2e-6 * max(abs(fd), 1e-3)


@pytest.fixture(scope="module")
def small():
    sh = W.shell_config(ncentre=2, seed=3)
    b = S.ShellBasis(sh.xyz, sh.lmn, sh.start, sh.exps, sh.coefs, sh.atom)
    return b, S.ShellPairs(b)


def test_unit_self_overlap(small):
    b, _ = small
    for f in range(b.nbf):
        assert abs(S.overlap(b, f, f) - 1.0) <= 1e-13
    # s overlap against the closed form
    s0 = [f for f in range(b.nbf) if not b.lmn[f].any()]
    f, g = s0[0], s0[-1]
    ref = 0.0
    for i in range(b.start[f], b.start[f + 1]):
        for j in range(b.start[g], b.start[g + 1]):
            a, c = b.exps[i], b.exps[j]
            r2 = ((b.xyz[f] - b.xyz[g]) ** 2).sum()
            ref += b.coefs[i] * b.coefs[j] * math.exp(-a * c / (a + c) * r2) * (math.pi / (a + c)) ** 1.5
    assert abs(S.overlap(b, f, g) - ref) <= 1e-14


def test_eightfold_symmetry_psd_and_schwarz(small):
    b, sp = small
    rng = np.random.default_rng(4)
    for _ in range(20):
        i, j, k, l = (int(x) for x in rng.integers(0, b.nbf, 4))
        v = S.eri(b, i, j, k, l)
        for p_ in ((j, i, k, l), (i, j, l, k), (k, l, i, j), (l, k, j, i)):
            assert abs(S.eri(b, *p_) - v) <= 1e-14 * max(1.0, abs(v))
    V = sp.matrix()
    ev = np.linalg.eigvalsh(V)
    assert ev.min() >= -1e-12 * ev.max()
    d = np.sqrt(np.diag(V))
    assert np.all(np.abs(V) <= np.outer(d, d) * (1 + 1e-12) + 1e-15)
