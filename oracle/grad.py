"""Implicit derivative of a converged quasiparticle energy.

At a root of f(w) = w - e_q - Sigma_qq(w) (Eq. qpapp), the implicit-function
theorem gives, for any parameter theta of e or of the Cholesky factors,

    dw/dtheta = P * (de_q/dtheta + dSigma_qq/dtheta |_w),
    P = 1 / (1 - dSigma/dw)                       (the pole strength, Eq. ps).

The paper does not differentiate; this is the derivative of its Eq. SE and
Eq. iter written out.  With X = (qx|sy) from Eq. aomo and each sum of Eq. SE
as sum n / D with n = (2 X_xy - X_yx) X_xy and D = w + e_s - e_x - e_y:

    dSigma/dX_xy = (4 X_xy - 2 X_yx) / D_xy          (D_xy = D_yx),
    dSigma/de_s = -sum n / D^2,  dSigma/de_x = +sum n / D^2 (x in either slot),

and X_xy = sum_K B^K_qx B^K_sy is bilinear in the factors.  The transform
B^K = C^T A^K C (Eq. transformation) chains the factor gradient to C.
"""
from __future__ import annotations

import numpy as np

from .ao2mo import unpack


def qp_gradient(Lq: np.ndarray, Lov: np.ndarray, eps: np.ndarray, nocc: int, q: int,
                w: float):
    """dw/d(eps, Lq, Lov) at a converged root w of orbital q.

    Lq [nmo, M] (row q of the factors), Lov [o, v, M].  Returns
    (d_eps [nmo], d_Lq [nmo, M], d_Lov [o, v, M], P)."""
    o, v, M = Lov.shape
    nmo = o + v
    eo, ev = eps[:nocc], eps[nocc:]
    Lq_occ, Lq_vir = Lq[:nocc], Lq[nocc:]
    Lov2 = Lov.reshape(o * v, M)
    d_eps = np.zeros(nmo)
    d_Lq = np.zeros((nmo, M))
    d_Lov = np.zeros((o, v, M))
    # first sum of Eq. SE: Y[i, j, a] = (qi|aj), D = w + e_a - e_i - e_j
    Y = (Lq_occ @ Lov2.T).reshape(o, o, v)
    Yx = Y.transpose(1, 0, 2)
    D1 = w + ev[None, None, :] - eo[:, None, None] - eo[None, :, None]
    n1 = (2 * Y - Yx) * Y
    G1 = (4 * Y - 2 * Yx) / D1
    r1 = n1 / D1 ** 2
    # second sum of Eq. SE: U[a, i, b] = (qa|ib), D = w + e_i - e_a - e_b
    U = (Lq_vir @ Lov2.T).reshape(v, o, v)
    Ux = U.transpose(2, 1, 0)
    D2 = w + eo[None, :, None] - ev[:, None, None] - ev[None, None, :]
    n2 = (2 * U - Ux) * U
    G2 = (4 * U - 2 * Ux) / D2
    r2 = n2 / D2 ** 2
    dsig = -(r1.sum() + r2.sum())
    P = 1.0 / (1.0 - dsig)
    # energy gradients of Sigma
    d_eps[nocc:] += -r1.sum(axis=(0, 1))                       # e_a in D1
    d_eps[:nocc] += r1.sum(axis=(1, 2)) + r1.sum(axis=(0, 2))  # e_i, e_j in D1
    d_eps[:nocc] += -r2.sum(axis=(0, 2))                       # e_i in D2
    d_eps[nocc:] += r2.sum(axis=(1, 2)) + r2.sum(axis=(0, 1))  # e_a, e_b in D2
    d_eps[q] += 1.0                                            # de_q/de_q
    # factor gradients of Sigma: Y = Lq_occ Lov2^T, U = Lq_vir Lov2^T
    G1m = G1.reshape(o, o * v)
    d_Lq[:nocc] = G1m @ Lov2
    d_Lov += (G1m.T @ Lq_occ).reshape(o, v, M)
    G2m = G2.reshape(v, o * v)
    d_Lq[nocc:] = G2m @ Lov2
    d_Lov += (G2m.T @ Lq_vir).reshape(o, v, M)
    return P * d_eps, P * d_Lq, P * d_Lov, P


def transform_gradient(L: np.ndarray, C: np.ndarray, nocc: int, orbitals: np.ndarray,
                       d_Lov: np.ndarray, d_Lp: np.ndarray) -> np.ndarray:
    """Chain d(.)/dLov [o, v, M] and d(.)/dLp [np, nmo, M] to d(.)/dC [nbf, nmo]
    through Lov^K = C_occ^T A^K C_vir and Lp^K[t] = C_{.,q_t}^T A^K C."""
    nbf, nmo = C.shape
    orbitals = np.asarray(orbitals)
    dC = np.zeros_like(C)
    Cocc, Cvir, Cp = C[:, :nocc], C[:, nocc:], C[:, orbitals]
    for K in range(L.shape[0]):
        A = unpack(L[K], nbf)
        gov = d_Lov[:, :, K]                      # [o, v]
        dC[:, :nocc] += A @ Cvir @ gov.T
        dC[:, nocc:] += A @ Cocc @ gov
        gp = d_Lp[:, :, K]                        # [np, nmo]
        dCp = A @ C @ gp.T                        # d/dC[:, q_t]
        for t, qt in enumerate(orbitals):
            dC[:, qt] += dCp[:, t]
        dC += A @ Cp @ gp
    return dC
