"""Newton quasiparticle solve of omega = e_q + Sigma_qq(omega).

Eq. qpapp is solved by Newton-Raphson (Eq. iter):
    w^(n+1) = w^(n) + (e_q + Sigma(w^(n)) - w^(n)) P^(n),
    P^(n)   = (1 - dSigma/dw |_(w^(n)))^(-1)            (Eq. ps),
starting from w^(0) = e_q and stopping when |w^(n+1) - w^(n)| <= Delta
(Eq. NR, Delta = 1e-5 in the paper).  Reported: w^(n+1), the pole strength
P^(n) of the last step, the number of Sigma evaluations, and a status
(0 converged, 1 not converged within max_iter, 2 non-finite iterate).
The iteration is plain Newton, as printed: no bracketing or damping.

``bracketed_qp`` is the safeguarded variant (not in the paper): every pole of
Sigma_qq lies at w = e_i + e_j - e_a or w = e_a + e_b - e_i, and between two
neighbouring poles f(w) = w - e_q - Sigma(w) is strictly increasing (every
residue is >= 0) and runs from -inf to +inf, so the interval around e_q holds
exactly one root.  The Newton step of Eq. iter is kept while it stays inside
the current bracket [lo, hi] of that root; otherwise the step bisects.
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


def pole_bracket(eps: np.ndarray, nocc: int, eps_q: float) -> tuple[float, float]:
    """The poles of Sigma (Eq. SE denominators) nearest to e_q below and above:
    every e_i + e_j - e_a and e_a + e_b - e_i (+-inf if none)."""
    eo, ev = eps[:nocc], eps[nocc:]
    poles = np.concatenate([(eo[:, None, None] + eo[None, :, None] - ev[None, None, :]).ravel(),
                            (ev[:, None, None] + ev[None, :, None] - eo[None, None, :]).ravel()])
    below, above = poles[poles < eps_q], poles[poles > eps_q]
    return (float(below.max()) if below.size else -np.inf,
            float(above.min()) if above.size else np.inf)


def bracketed_qp(sigma: Callable[[float], tuple[float, float]], eps_q: float, lo: float,
                 hi: float, conv: float = 1e-5, max_iter: int = 100
                 ) -> tuple[float, float, int, int]:
    """Safeguarded Newton inside the pole-free interval (lo, hi) around e_q.

    From w = e_q: evaluate f = w - e_q - Sigma(w) and f' = 1 - dSigma/dw; the
    sign of f moves lo (f < 0) or hi (f > 0) to w; the next iterate is the
    Newton step w - f/f' if it lies strictly inside (lo, hi), else the
    midpoint.  Stops when the step is <= conv.  Returns (omega, pole strength
    1/f' at the last evaluation, evaluations, status).  A side with no pole
    (+-inf) is taken 10 Ha beyond e_q."""
    lo = lo if np.isfinite(lo) else eps_q - 10.0
    hi = hi if np.isfinite(hi) else eps_q + 10.0
    w = float(eps_q)
    P = 1.0
    for n in range(1, max_iter + 1):
        s, ds = sigma(w)
        f, fp = w - eps_q - s, 1.0 - ds
        P = 1.0 / fp
        if f < 0:
            lo = w
        else:
            hi = w
        w_new = w - f / fp
        if not (lo < w_new < hi):
            w_new = 0.5 * (lo + hi)
        if not np.isfinite(w_new):
            return w_new, P, n, QP_NONFINITE
        if abs(w_new - w) <= conv:
            return w_new, P, n, QP_OK
        w = w_new
    return w, P, max_iter, QP_NO_CONVERGENCE
