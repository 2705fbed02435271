"""Diagonal second-order self-energy Sigma(2)_qq(omega) and its derivative.

Eq. SE (spatial orbitals, i, j occupied; a, b virtual):

  Sigma_qq(w) = sum_{i,j,a} (2(qi|aj) - (qj|ai)) (qi|aj) / (w + e_a - e_i - e_j)
              + sum_{i,a,b} (2(qa|ib) - (qb|ia)) (qa|ib) / (w + e_i - e_a - e_b)

with the MO integrals recomputed from the Cholesky factors by Eq. aomo at
every evaluation, as the paper does in its Newton iterations (Sec. III).
The pole strength of Eq. ps needs dSigma/dw, taken analytically:
dSigma/dw = - sum numerator / denominator^2.

``mp2_from_factors`` is Eq. MP2 on the same factors (the correlation energy
the paper sets beside Eq. SE).  ``sigma2_spin_orbital`` and ``mp2_energy``
are independent formulations (spin-orbital antisymmetrised integrals; Eq. MP2
from explicit MO integrals) used only as pins.
"""
from __future__ import annotations

import numpy as np


def sigma2_from_factors(Lq: np.ndarray, Lov: np.ndarray, eps: np.ndarray,
                        nocc: int, E: np.ndarray, parts: bool = False):
    """Sigma_qq(E) and dSigma_qq/dE for one orbital q at every E (Eq. SE).

    Lq  [nmo, M]   : B^K_{q r} for all MOs r (row q of the factors)
    Lov [o, v, M]  : B^K_{i a}
    E   [nE]
    With ``parts=True`` the two sums of Eq. SE are returned separately as
    (first_sum, second_sum), each [nE], instead of (Sigma, dSigma).
    """
    E = np.atleast_1d(np.asarray(E, dtype=np.float64))
    o, v = Lov.shape[0], Lov.shape[1]
    eo, ev = eps[:nocc], eps[nocc:]
    Lq_occ, Lq_vir = Lq[:nocc], Lq[nocc:]
    Lov2 = Lov.reshape(o * v, -1)                      # row i*v + a
    # first sum: (qi|aj) = sum_K B^K_qi B^K_aj, stored as Y[i, j, a]
    Y = (Lq_occ @ Lov2.T).reshape(o, o, v)
    num1 = (2.0 * Y - Y.transpose(1, 0, 2)) * Y        # (qj|ai) = Y[j, i, a]
    den1 = ev[None, None, :] - eo[:, None, None] - eo[None, :, None]
    # second sum: (qa|ib) = sum_K B^K_qa B^K_ib, stored as U[a, i, b]
    U = (Lq_vir @ Lov2.T).reshape(v, o, v)
    num2 = (2.0 * U - U.transpose(2, 1, 0)) * U        # (qb|ia) = U[b, i, a]
    den2 = eo[None, :, None] - ev[:, None, None] - ev[None, None, :]
    s1 = np.empty(E.shape[0])
    s2 = np.empty(E.shape[0])
    dsig = np.empty(E.shape[0])
    for k, w in enumerate(E):
        d1 = w + den1
        d2 = w + den2
        s1[k] = (num1 / d1).sum()
        s2[k] = (num2 / d2).sum()
        dsig[k] = -(num1 / d1 ** 2).sum() - (num2 / d2 ** 2).sum()
    if parts:
        return s1, s2
    return s1 + s2, dsig


def sigma2_from_mo_integrals(g: np.ndarray, eps: np.ndarray, nocc: int, q: int,
                             E: np.ndarray) -> np.ndarray:
    """Eq. SE with explicit MO integrals g[p,q,r,s] = (pq|rs) (small cases)."""
    E = np.atleast_1d(np.asarray(E, dtype=np.float64))
    nmo = g.shape[0]
    occ = np.arange(nocc)
    vir = np.arange(nocc, nmo)
    out = np.zeros(E.shape[0])
    for k, w in enumerate(E):
        s = 0.0
        for i in occ:
            for j in occ:
                for a in vir:
                    s += (2 * g[q, i, a, j] - g[q, j, a, i]) * g[q, i, a, j] / (
                        w + eps[a] - eps[i] - eps[j])
        for i in occ:
            for a in vir:
                for b in vir:
                    s += (2 * g[q, a, i, b] - g[q, b, i, a]) * g[q, a, i, b] / (
                        w + eps[i] - eps[a] - eps[b])
        out[k] = s
    return out


def sigma2_spin_orbital(g: np.ndarray, eps: np.ndarray, nocc: int, q: int,
                        w: float) -> float:
    """Second-order self-energy in a spin-orbital basis, spin q = alpha.

    Sigma_qq = 1/2 sum_{i,a,b} |<ab||qi>|^2 / (w + e_i - e_a - e_b)
             + 1/2 sum_{i,j,a} |<ij||qa>|^2 / (w + e_a - e_i - e_j),
    <pq||rs> = <pq|rs> - <pq|sr>,  <pq|rs> = (pr|qs) * [spins match].
    Spin sums are done by brute force over explicit spin labels.
    """
    nmo = g.shape[0]
    so = [(p, s) for p in range(nmo) for s in (0, 1)]

    def phys(p, qq, r, t):
        (P, sp), (Q, sq), (R, sr), (T, st) = p, qq, r, t
        return g[P, R, Q, T] if (sp == sr and sq == st) else 0.0

    def anti(p, qq, r, t):
        return phys(p, qq, r, t) - phys(p, qq, t, r)

    qs = (q, 0)
    occ = [x for x in so if x[0] < nocc]
    vir = [x for x in so if x[0] >= nocc]
    s = 0.0
    for i in occ:
        for a in vir:
            for b in vir:
                s += 0.5 * anti(a, b, qs, i) ** 2 / (w + eps[i[0]] - eps[a[0]] - eps[b[0]])
    for i in occ:
        for j in occ:
            for a in vir:
                s += 0.5 * anti(i, j, qs, a) ** 2 / (w + eps[a[0]] - eps[i[0]] - eps[j[0]])
    return s


def mp2_from_factors(Lov: np.ndarray, eps: np.ndarray, nocc: int, pairs: bool = False,
                     rows=None):
    """MP2 correlation energy, Eq. MP2, with (ai|bj) = sum_K B^K_ia B^K_jb
    recomputed from the factors (Eq. aomo).

    Lov [o, v, M].  For each occupied i the integrals of all (j, a, b) come
    from one matrix product, X[a, j, b] = (ia|jb); the exchange integral
    (aj|bi) = (ib|ja) is X[b, j, a].  With ``pairs=True`` returns the per-i
    sums e_i = sum_{j,a,b} (...) [o] instead of their total; ``rows`` limits
    them to a subset of i (then only those e_i are returned)."""
    o, v, M = Lov.shape
    eo, ev = eps[:nocc], eps[nocc:]
    Lov2 = Lov.reshape(o * v, M)
    idx = range(o) if rows is None else [int(i) for i in rows]
    e = np.zeros(len(idx))
    for n, i in enumerate(idx):
        X = (Lov[i] @ Lov2.T).reshape(v, o, v)
        Xx = X.transpose(2, 1, 0)
        D = eo[i] + eo[None, :, None] - ev[:, None, None] - ev[None, None, :]
        e[n] = ((2 * X - Xx) * X / D).sum()
    if rows is not None:
        return e
    return e if pairs else float(e.sum())


def mp2_energy(g: np.ndarray, eps: np.ndarray, nocc: int) -> float:
    """MP2 correlation energy, Eq. MP2, from explicit MO integrals."""
    nmo = g.shape[0]
    s = 0.0
    for i in range(nocc):
        for j in range(nocc):
            for a in range(nocc, nmo):
                for b in range(nocc, nmo):
                    s += (2 * g[a, i, b, j] - g[a, j, b, i]) * g[a, i, b, j] / (
                        eps[i] + eps[j] - eps[a] - eps[b])
    return s
