"""Product densities and electron-repulsion integrals over s-type Gaussians.

Sec. II.A defines the product-density set rho_I = chi_mu chi_nu with
I = (mu, nu), mu <= nu, and the ERI (mu nu|lambda sigma) = (rho_I|V|rho_J)
(Eq. integral).  For normalised s-type primitives
chi_mu(r) = (2 a_mu/pi)^(3/4) exp(-a_mu |r - A_mu|^2) the integral has the
textbook closed form

    (rho_I|rho_J) = 2 pi^(5/2) / (p q sqrt(p+q)) * K_I K_J * F0(T),
    p = a_mu + a_nu,  P = (a_mu A_mu + a_nu A_nu)/p,
    K_I = N_mu N_nu exp(-a_mu a_nu |A_mu - A_nu|^2 / p),
    T = p q/(p+q) |P - Q|^2,  F0(T) = (1/2) sqrt(pi/T) erf(sqrt(T)).

Packed pair index (the paper leaves the order open): I = nu(nu+1)/2 + mu for
0 <= mu <= nu < N, i.e. pairs ordered by nu, then mu.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

TWO_PI_5_2 = 2.0 * math.pi ** 2.5


def pair_index(mu, nu):
    """Packed index of the pair (mu, nu) with mu <= nu (either order accepted)."""
    mu = np.asarray(mu)
    nu = np.asarray(nu)
    lo = np.minimum(mu, nu)
    hi = np.maximum(mu, nu)
    return hi * (hi + 1) // 2 + lo


def pair_list(nbf: int) -> tuple[np.ndarray, np.ndarray]:
    """(mu[I], nu[I]) for I = 0 .. N(N+1)/2 - 1 in packed order."""
    nu, mu = [], []
    for n in range(nbf):
        for m in range(n + 1):
            mu.append(m)
            nu.append(n)
    return np.array(mu, dtype=np.int64), np.array(nu, dtype=np.int64)


def boys_f0(T):
    """F0(T) = int_0^1 exp(-T u^2) du = (1/2) sqrt(pi/T) erf(sqrt(T)).

    For T < 1e-10 the two-term series 1 - T/3 is used (error < T^2/10)."""
    T = np.asarray(T, dtype=np.float64)
    small = T < 1e-10
    Ts = np.where(small, 1.0, T)
    x = np.sqrt(Ts)
    big = 0.5 * math.sqrt(math.pi) * erf(x) / x
    return np.where(small, 1.0 - T / 3.0, big)


class PairData:
    """Gaussian-product data of every product density rho_I (Sec. II.A)."""

    def __init__(self, xyz: np.ndarray, alpha: np.ndarray):
        xyz = np.asarray(xyz, dtype=np.float64)
        alpha = np.asarray(alpha, dtype=np.float64)
        self.nbf = alpha.shape[0]
        self.mu, self.nu = pair_list(self.nbf)
        am, an = alpha[self.mu], alpha[self.nu]
        A, B = xyz[self.mu], xyz[self.nu]
        norm = (2.0 * alpha / math.pi) ** 0.75
        self.p = am + an
        self.P = (am[:, None] * A + an[:, None] * B) / self.p[:, None]
        r2 = ((A - B) ** 2).sum(axis=1)
        self.K = norm[self.mu] * norm[self.nu] * np.exp(-am * an / self.p * r2)

    @property
    def npair(self) -> int:
        return self.p.shape[0]


def eri_from_pairs(pd: PairData, I, J):
    """(rho_I|rho_J) for index arrays I, J (broadcast), Eq. integral."""
    p, q = pd.p[I], pd.p[J]
    d2 = ((pd.P[I] - pd.P[J]) ** 2).sum(axis=-1)
    T = p * q / (p + q) * d2
    return TWO_PI_5_2 / (p * q * np.sqrt(p + q)) * pd.K[I] * pd.K[J] * boys_f0(T)


def eri_diagonal(pd: PairData) -> np.ndarray:
    """D_I = (rho_I|rho_I) for every pair: the initial residual diagonal."""
    I = np.arange(pd.npair)
    return eri_from_pairs(pd, I, I)


def eri_column(pd: PairData, J: int) -> np.ndarray:
    """Column J of the supermatrix: (rho_I|rho_J) for all I."""
    I = np.arange(pd.npair)
    return eri_from_pairs(pd, I, np.full_like(I, J))


def eri_matrix(pd: PairData) -> np.ndarray:
    """The explicit supermatrix V_IJ = (rho_I|rho_J) (small bases only)."""
    n = pd.npair
    I = np.arange(n)
    V = np.empty((n, n))
    for J in range(n):
        V[:, J] = eri_from_pairs(pd, I, np.full(n, J))
    return V


def eri_tensor(pd: PairData) -> np.ndarray:
    """Full 4-index (mu nu|lambda sigma) from the supermatrix (tiny bases)."""
    N = pd.nbf
    V = eri_matrix(pd)
    idx = pair_index(np.arange(N)[:, None], np.arange(N)[None, :])
    return V[idx[:, :, None, None], idx[None, None, :, :]]
