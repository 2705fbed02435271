"""Pins for the atomic Cholesky basis and its V-approximation (oracle/acd.py).

* the basis holds one-centre densities only, the same local choice for every
  atom of a type, and each type's choice is the pivot set of the isolated
  atom's decomposition;
* with the full decomposition's pivots as the basis, the V-approximation
  reproduces that decomposition's L^T L (the pivoted Cholesky factor is the
  Nystrom approximation on its pivots): ties ri_factors to the pinned CD;
* the approximation is exact on every basis density (rows of V);
* Eq. error_approx: the error matrix V - B^T B is positive semidefinite;
* the strict bound of the isolated atoms carries over: every one-centre
  density's error is <= delta (more fitting densities can only lower it).
"""
import numpy as np
import pytest

import workloads as W
from oracle import acd, cd, eri


@pytest.fixture(scope="module", params=[("c0", 1e-6), ("c0", 1e-3)])
def case(request):
    name, delta = request.param
    m = W.config0()
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    V = eri.eri_matrix(pd)
    aux = acd.aux_pairs(m.basis.alpha, m.basis.atom, delta)
    B = acd.ri_factors(pd, aux)
    return m, pd, V, aux, B, delta


def test_basis_is_one_centre_and_per_type(case):
    m, pd, V, aux, B, delta = case
    at = m.basis.atom
    assert np.all(at[pd.mu[aux]] == at[pd.nu[aux]])
    types = acd.atom_types(m.basis.alpha, at)
    assert len(types) == 1                      # every centre carries the same exponents
    per_atom = [aux[at[pd.mu[aux]] == a] for a in np.unique(at)]
    first = np.flatnonzero(at == 0)
    loc0 = [(int(np.searchsorted(first, pd.mu[P])), int(np.searchsorted(first, pd.nu[P])))
            for P in per_atom[0]]
    assert loc0 == [tuple(sorted(x)) for x in acd.atomic_pivots(list(types)[0], delta)]
    assert len({len(x) for x in per_atom}) == 1


def test_full_cd_pivots_reproduce_the_cd_factor():
    m = W.config0()
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    res = cd.decompose(pd, 1e-5)
    B = acd.ri_factors(pd, res.piv)
    scale = res.scale
    assert np.abs(B.T @ B - res.L.T @ res.L).max() <= 1e-10 * scale


def test_exact_on_basis_densities(case):
    m, pd, V, aux, B, delta = case
    approx = B.T @ B
    assert np.abs(approx[aux] - V[aux]).max() <= 1e-11 * np.abs(V).max()


def test_error_matrix_is_positive_semidefinite(case):
    m, pd, V, aux, B, delta = case
    Dm = V - B.T @ B
    ev = np.linalg.eigvalsh(0.5 * (Dm + Dm.T))
    assert ev.min() >= -1e-10 * np.abs(V).max()


def test_one_centre_error_within_delta(case):
    m, pd, V, aux, B, delta = case
    at = m.basis.atom
    one = at[pd.mu] == at[pd.nu]
    diag = np.diag(V - B.T @ B)
    assert diag[one].max() <= delta * (1 + 1e-9)
