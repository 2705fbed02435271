"""Atomic Cholesky basis and the V-approximation built on it (test
infrastructure: imported only by tests/, __graft_entry__.smoke() and the CPU
legs of bench.py; shares no code with the CUDA path).

Sec. II.A, atomic CD: the Cholesky basis holds only one-centre product
densities, chosen once per unique atom / AO basis pair.  Here a unique atom
is a set of functions with the same exponents on one centre; its basis is the
pivot set of the threshold-delta Cholesky decomposition (cd.decompose, the
same pivot rule as the full CD) of the isolated atom's one-centre ERI matrix.
Every atom of the molecule contributes its type's pivots, as densities on its
own centre.  The ERIs then follow the V-approximation of Eq. int_approx,

    (rho_I|rho_J) ~ sum_{K,L} (rho_I|rho~_K) [V^-1]_{KL} (rho~_L|rho_J),

with V the Coulomb metric of the basis densities.  With V = L_m L_m^T
(Cholesky), B = L_m^-1 (rho~|rho_I) gives the same factor form as Eq. CD,
(rho_I|rho_J) ~ sum_K B^K_I B^K_J, and Eq. error_approx says the error
matrix D = V - B^T B is positive semidefinite.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cholesky, solve_triangular

from . import cd, eri


def atom_types(alpha: np.ndarray, atom: np.ndarray) -> dict:
    """{exponent tuple: [atoms]} in order of first appearance; the functions of
    each atom are taken in their basis order."""
    types: dict = {}
    for a in np.unique(atom):
        key = tuple(float(x) for x in alpha[atom == a])
        types.setdefault(key, []).append(int(a))
    return types


def atomic_pivots(alpha_atom, delta: float) -> list[tuple[int, int]]:
    """Local (mu, nu) of the one-centre densities the isolated atom's
    decomposition selects, in pivot order."""
    a = np.asarray(alpha_atom, dtype=np.float64)
    pd = eri.PairData(np.zeros((a.size, 3)), a)
    res = cd.decompose(pd, delta)
    return [(int(pd.mu[P]), int(pd.nu[P])) for P in res.piv]


def aux_pairs(alpha: np.ndarray, atom: np.ndarray, delta: float) -> np.ndarray:
    """Packed molecule pair indices of the atomic Cholesky basis: for each atom
    (ascending centre index) its type's pivots on its own functions."""
    alpha = np.asarray(alpha)
    atom = np.asarray(atom)
    piv_of = {key: atomic_pivots(key, delta) for key in atom_types(alpha, atom)}
    out = []
    for a in np.unique(atom):
        funcs = np.flatnonzero(atom == a)
        key = tuple(float(x) for x in alpha[funcs])
        for mu, nu in piv_of[key]:
            out.append(int(eri.pair_index(funcs[mu], funcs[nu])))
    return np.array(out, dtype=np.int64)


def ri_factors(pd: eri.PairData, aux: np.ndarray) -> np.ndarray:
    """B [naux, npair] with B^T B the V-approximation (Eq. int_approx) over the
    basis densities aux."""
    cols = np.stack([eri.eri_column(pd, int(P)) for P in aux])   # (rho~_K|rho_I)
    V = cols[:, aux]                                             # metric (rho~_K|rho~_L)
    Lm = cholesky(V, lower=True)
    return solve_triangular(Lm, cols, lower=True)
