"""Threshold-delta diagonal-pivoted Cholesky decomposition of the ERI supermatrix.

Sec. II.A builds the Cholesky basis by Gram-Schmidt in the Coulomb metric
(Eq. gs_coulomb): the K-th basis density is the K-th chosen product density
minus its projections on the earlier ones, divided by sqrt(n_K), where n_K is
the Coulomb self-repulsion left after those projections.  The integral table
L^K_J = (rho_J|V|rho~_K) (Eq. CD) then satisfies

    L^K_J = [ (rho_J|rho_P) - sum_{I<K} L^I_J L^I_P ] / sqrt(n_K),
    n_K   = D_P,   D_J = (rho_J|rho_J) - sum_{I<=K} (L^I_J)^2,

with P the density chosen at step K and D the residual diagonal (the error
D_JJ of Eq. error_approx).  The paper delegates the pivot rule to the
"modified Cholesky" algorithm; the readings taken here are:

* pivot: the largest residual diagonal among the candidates; candidates
  within ``tie_rel * max(D at start)`` of that maximum (and above delta_eff)
  count as tied and the lowest packed index wins;
* stop: as soon as every candidate residual is <= delta_eff
  (delta_eff = max(delta, npair * eps_mach * max(D at start))), so the strict
  bound D_JJ <= delta of Eq. stricterr holds on the candidate set;
* after a density is chosen its own residual is set to exactly zero (it is
  represented exactly, Sec. II.A);
* full scheme: every pair is a candidate; atomic scheme: only one-centre
  pairs (mu and nu on the same centre) are candidates (Sec. II.A, atomic CD),
  while L is still formed for every pair.
"""
from __future__ import annotations

from typing import Callable, Optional

import numpy as np

from .eri import PairData, eri_column, eri_diagonal

EPS = np.finfo(np.float64).eps
TIE_REL = 1e-12
NOT_PD_REL = 1e-10


class RankCapError(RuntimeError):
    """More than max_rank Cholesky vectors would be needed."""


class NotPositiveDefiniteError(RuntimeError):
    """A residual diagonal went below -1e-10 * max(D at start)."""


class CDResult:
    def __init__(self, L, piv, D, delta_eff, scale):
        self.L = L            # [M, npair] float64, L[K, I] = L^K_I
        self.piv = piv        # [M] int64, packed index chosen at step K
        self.D = D            # [npair] residual diagonal after the last step
        self.delta_eff = delta_eff
        self.scale = scale    # max initial diagonal

    @property
    def M(self) -> int:
        return int(self.piv.shape[0])


def candidate_mask(pd: PairData, atom: Optional[np.ndarray], scheme: str) -> np.ndarray:
    if scheme == "full":
        return np.ones(pd.npair, dtype=bool)
    if scheme == "atomic":
        atom = np.asarray(atom)
        return atom[pd.mu] == atom[pd.nu]
    raise ValueError(f"unknown scheme {scheme!r}")


def effective_delta(delta: float, npair: int, scale: float) -> float:
    return max(float(delta), npair * EPS * scale)


def select_pivot(D: np.ndarray, cand: np.ndarray, scale: float, delta_eff: float,
                 tie_rel: float = TIE_REL) -> tuple[int, float]:
    """Largest candidate residual G (clamped at 0) and the pivot: the lowest
    candidate index whose residual is >= G - tie_rel*scale and > delta_eff.
    The pivot is meaningful only when G > delta_eff."""
    Dc = np.where(cand, np.maximum(D, 0.0), -np.inf)
    G = float(Dc.max())
    ok = (Dc >= G - tie_rel * scale) & (Dc > delta_eff)
    P = int(np.flatnonzero(ok)[0]) if ok.any() else int(np.argmax(Dc))
    return P, G


def decompose(pd: PairData, delta: float, scheme: str = "full",
              atom: Optional[np.ndarray] = None, max_rank: Optional[int] = None,
              column: Optional[Callable[[int], np.ndarray]] = None,
              tie_rel: float = TIE_REL, diagonal: Optional[np.ndarray] = None) -> CDResult:
    """Cholesky vectors L^K (Eq. CD) by Gram-Schmidt steps (Eq. gs_coulomb).

    ``column(P)`` returns (rho_I|rho_P) for all I; by default it is computed
    on the fly from the closed-form integral.  Pass ``lambda P: V[:, P]`` to
    decompose an explicit supermatrix.  ``diagonal`` (the (rho_I|rho_I)) goes
    with a ``column`` of another basis (contracted shells); ``pd`` then only
    supplies npair and the pair list (mu, nu) for the atomic candidate set.
    """
    n = pd.npair
    if column is None:
        def column(P):
            return eri_column(pd, P)
    if max_rank is None:
        max_rank = n
    cand = candidate_mask(pd, atom, scheme)
    D = eri_diagonal(pd) if diagonal is None else np.array(diagonal, dtype=np.float64)
    scale = float(D.max())
    delta_eff = effective_delta(delta, n, scale)
    L = np.zeros((min(max_rank, n, 256), n))
    piv: list[int] = []
    k = 0
    while True:
        if not np.all(np.isfinite(D)) or D.min() < -NOT_PD_REL * scale:
            raise NotPositiveDefiniteError(f"residual diagonal {D.min():.3e} at step {k}")
        P, G = select_pivot(D, cand, scale, delta_eff, tie_rel)
        if G <= delta_eff:
            break
        if k >= max_rank:
            raise RankCapError(f"rank cap {max_rank} reached with max residual {G:.3e}")
        if k == L.shape[0]:
            L = np.concatenate([L, np.zeros((min(L.shape[0], n - k), n))])
        nK = D[P]
        # projections of rho_J on the earlier basis densities, Eq. gs_coulomb
        proj = L[:k].T @ L[:k, P] if k else np.zeros(n)
        L[k] = (column(P) - proj) / np.sqrt(nK)
        D = D - L[k] ** 2
        D[P] = 0.0
        piv.append(P)
        k += 1
    return CDResult(L[:k].copy(), np.array(piv, dtype=np.int64), D, delta_eff, scale)


def reconstruct(L: np.ndarray) -> np.ndarray:
    """Approximate supermatrix sum_K L^K_I L^K_J (Eq. CD)."""
    return L.T @ L
