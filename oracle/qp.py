"""Newton quasiparticle solve of omega = e_q + Sigma_qq(omega).

Eq. qpapp is solved by Newton-Raphson (Eq. iter):
    w^(n+1) = w^(n) + (e_q + Sigma(w^(n)) - w^(n)) P^(n),
    P^(n)   = (1 - dSigma/dw |_(w^(n)))^(-1)            (Eq. ps),
starting from w^(0) = e_q and stopping when |w^(n+1) - w^(n)| <= Delta
(Eq. NR, Delta = 1e-5 in the paper).  Reported: w^(n+1), the pole strength
P^(n) of the last step, the number of Sigma evaluations, and a status
(0 converged, 1 not converged within max_iter, 2 non-finite iterate).
The iteration is plain Newton, as printed: no bracketing or damping.
"""
from __future__ import annotations

from typing import Callable

import numpy as np

QP_OK = 0
QP_NO_CONVERGENCE = 1
QP_NONFINITE = 2


def newton_qp(sigma: Callable[[float], tuple[float, float]], eps_q: float,
              conv: float = 1e-5, max_iter: int = 50) -> tuple[float, float, int, int]:
    """Returns (omega, pole_strength, iterations, status)."""
    w = float(eps_q)
    P = 1.0
    for n in range(1, max_iter + 1):
        s, ds = sigma(w)
        P = 1.0 / (1.0 - ds)
        w_new = w + (eps_q + s - w) * P
        if not np.isfinite(w_new):
            return w_new, P, n, QP_NONFINITE
        if abs(w_new - w) <= conv:
            return w_new, P, n, QP_OK
        w = w_new
    return w, P, max_iter, QP_NO_CONVERGENCE
