"""Pins for the oracle's Cholesky decomposition (Sec. II.A, Eq. CD, Eq. stricterr).

What the paper fixes and what the mathematics fixes, checked against the
explicit supermatrix:
* strict error bound |V - L^T L| <= delta (Eq. stricterr, via Schwarz);
* pivot pairs reproduced to machine precision (Sec. II.A, exactness);
* the pivot block of L is the LAPACK Cholesky factor of V[piv, piv], and the
  remaining rows solve L = V[:, piv] R^-T (an independent algorithm);
* delta = 0 reconstructs V to roundoff with rank <= N(N+1)/2 (continuity);
* the error falls and the rank grows monotonically as delta shrinks;
* each pivot is the largest residual diagonal, recomputed from scratch;
* the atomic scheme pivots on one-centre pairs only and bounds that block.
"""
import numpy as np
import pytest

import workloads as W
from oracle import cd, eri


@pytest.fixture(scope="module")
def c0():
    m = W.config0()
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    return m, pd, eri.eri_matrix(pd)


@pytest.mark.parametrize("delta", [1e-2, 1e-4, 1e-6, 1e-8])
def test_strict_error_bound(c0, delta):
    m, pd, V = c0
    r = cd.decompose(pd, delta)
    err = V - cd.reconstruct(r.L)
    assert np.abs(err).max() <= delta
    # the residual diagonal tracked by the algorithm is the true error diagonal
    np.testing.assert_allclose(r.D, np.diag(err), rtol=0, atol=1e-13 * r.scale)


def test_pivot_pairs_exact_and_lapack_factor(c0):
    m, pd, V = c0
    r = cd.decompose(pd, 1e-6)
    piv = r.piv
    approx = cd.reconstruct(r.L)
    assert np.abs((V - approx)[np.ix_(piv, piv)]).max() <= 1e-13 * r.scale
    R = np.linalg.cholesky(V[np.ix_(piv, piv)])          # LAPACK, lower
    np.testing.assert_allclose(r.L[:, piv].T, R, rtol=0, atol=1e-12)
    full = np.linalg.solve(R, V[piv, :]).T                 # V[:, piv] R^-T
    np.testing.assert_allclose(r.L.T, full, rtol=0, atol=1e-10)


def test_pivot_block_lower_triangular(c0):
    m, pd, V = c0
    r = cd.decompose(pd, 1e-6)
    blk = r.L[:, r.piv]            # blk[K, J] = L^K at pivot J
    upper = np.triu(blk.T, 1)      # entries L^K_{P_J} with K > J
    assert np.abs(upper).max() <= 1e-12


def test_delta_zero_exact_reconstruction(c0):
    m, pd, V = c0
    r = cd.decompose(pd, 0.0)
    assert r.M <= pd.npair
    assert np.abs(V - cd.reconstruct(r.L)).max() <= 1e-12
    assert r.delta_eff == pytest.approx(pd.npair * np.finfo(float).eps * r.scale)


def test_monotone_in_delta(c0):
    m, pd, V = c0
    errs, ranks = [], []
    for delta in [1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-10]:
        r = cd.decompose(pd, delta)
        errs.append(np.abs(V - cd.reconstruct(r.L)).max())
        ranks.append(r.M)
    assert all(b <= a for a, b in zip(errs, errs[1:]))
    assert all(b >= a for a, b in zip(ranks, ranks[1:]))


def test_each_pivot_is_argmax_of_fresh_residual(c0):
    m, pd, V = c0
    r = cd.decompose(pd, 1e-6)
    for k, P in enumerate(r.piv):
        D = np.diag(V) - (r.L[:k] ** 2).sum(axis=0)
        D[r.piv[:k]] = 0.0
        assert D[P] >= D.max() - 1e-12 * r.scale - 1e-14


def test_explicit_and_on_the_fly_columns_agree(c0):
    m, pd, V = c0
    a = cd.decompose(pd, 1e-6)
    b = cd.decompose(pd, 1e-6, column=lambda P: V[:, P])
    assert np.array_equal(a.piv, b.piv)
    np.testing.assert_allclose(a.L, b.L, rtol=0, atol=1e-14)


def test_atomic_scheme(c0):
    m, pd, V = c0
    atom = m.basis.atom
    r = cd.decompose(pd, 1e-6, scheme="atomic", atom=atom)
    one = atom[pd.mu] == atom[pd.nu]
    assert np.all(one[r.piv])
    err = V - cd.reconstruct(r.L)
    assert np.abs(err[np.ix_(one, one)]).max() <= 1e-6
    full = cd.decompose(pd, 1e-6)
    assert r.M < full.M


def test_rank_cap_raises(c0):
    m, pd, V = c0
    with pytest.raises(cd.RankCapError):
        cd.decompose(pd, 1e-6, max_rank=10)


def test_planted_sign_error_is_caught(c0, monkeypatch):
    """A plausible slip (an integral column off by one part in 1e9) must
    break the LAPACK-factor pin above."""
    m, pd, V = c0
    good = cd.decompose(pd, 1e-4)
    orig = cd.eri_column

    def bad_column(pd_, P):
        return orig(pd_, P) * (1 + 1e-9)
    monkeypatch.setattr(cd, "eri_column", bad_column)
    bad = cd.decompose(pd, 1e-4)
    R = np.linalg.cholesky(V[np.ix_(bad.piv, bad.piv)])
    assert np.abs(bad.L[:, bad.piv].T - R).max() > 1e-12 or not np.array_equal(bad.piv, good.piv)
