"""AO -> MO transform of the Cholesky vectors.

Eq. transformation: B^K_pq = sum_{mu,nu} C_{mu p} A^K_{mu nu} C_{nu q}, with
A^K the (symmetric) integral table L^K unpacked from the packed pair index.
Eq. aomo: (pq|rs) = sum_K B^K_pq B^K_rs.

Output blocks used by the self-energy (the paper recomputes MO integrals
from these factors in every Newton iteration, Sec. III):

* ``Lov[i, a, K] = B^K_{i, nocc+a}``  (occupied x virtual),
* ``Lp[t, r, K]  = B^K_{orbitals[t], r}`` (rows of the requested orbitals).
"""
from __future__ import annotations

import numpy as np

from .eri import pair_index


def unpack(Lk: np.ndarray, nbf: int) -> np.ndarray:
    """Symmetric N x N matrix A^K_{mu nu} from the packed vector L^K_I."""
    idx = pair_index(np.arange(nbf)[:, None], np.arange(nbf)[None, :])
    return Lk[idx]


def transform_full(L: np.ndarray, C: np.ndarray) -> np.ndarray:
    """B[K] = C^T A^K C for every K (Eq. transformation); [M, nmo, nmo]."""
    nbf = C.shape[0]
    out = np.empty((L.shape[0], C.shape[1], C.shape[1]))
    for K in range(L.shape[0]):
        out[K] = C.T @ unpack(L[K], nbf) @ C
    return out


def mo_factors(L: np.ndarray, C: np.ndarray, nocc: int,
               orbitals: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(Lov [o, v, M], Lp [np, nmo, M]) by Eq. transformation, one K at a time."""
    nbf, nmo = C.shape
    M = L.shape[0]
    orbitals = np.asarray(orbitals)
    Lov = np.empty((nocc, nmo - nocc, M))
    Lp = np.empty((orbitals.shape[0], nmo, M))
    Cocc, Cvir, Cp = C[:, :nocc], C[:, nocc:], C[:, orbitals]
    for K in range(M):
        A = unpack(L[K], nbf)
        Lov[:, :, K] = Cocc.T @ A @ Cvir
        Lp[:, :, K] = Cp.T @ A @ C
    return Lov, Lp


def mo_integrals(B: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum_K B^K_pq B^K_rs (Eq. aomo); [nmo]*4, tiny cases only."""
    return np.einsum("kpq,krs->pqrs", B, B)


def ao_to_mo_4index(eri4: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Conventional O(N^5) four-index transform of explicit AO integrals."""
    t = np.einsum("mnls,mp->pnls", eri4, C)
    t = np.einsum("pnls,nq->pqls", t, C)
    t = np.einsum("pqls,lr->pqrs", t, C)
    return np.einsum("pqrs,st->pqrt", t, C)
