"""Electron-repulsion integrals over contracted Cartesian Gaussians (s, p, d).

The paper's basis sets are contracted Gaussian shells with higher angular
momentum (Sec. III, cc-pVXZ); Eq. integral is the same Coulomb integral over
their products.  A basis function here is a normalised contraction on one
centre A,

    chi(r) = sum_k c_k x_A^l y_A^m z_A^n exp(-a_k |r - A|^2),   (x_A = x - A_x, ...)

with l + m + n = 0 (s), 1 (p: x, y, z) or 2 (Cartesian d: xx, xy, xz, yy,
yz, zz), the coefficients c_k carrying the normalisation of the whole
function (unit self-overlap).

Integrals follow the McMurchie-Davidson scheme, written from its defining
relations.  The product of two 1-D Cartesian Gaussians with exponents a, b
on centres A, B is a finite sum of Hermite Gaussians about P = (aA + bB)/p,
p = a + b,

    x_A^i x_B^j exp(-a x_A^2 - b x_B^2) = sum_t E_t^{ij} Lambda_t(x; p, P),
    E_0^{00} = exp(-a b / p (A - B)^2),
    E_t^{i+1,j} = E_{t-1}^{ij} / (2p) + (P - A) E_t^{ij} + (t + 1) E_{t+1}^{ij},
    E_t^{i,j+1} = E_{t-1}^{ij} / (2p) + (P - B) E_t^{ij} + (t + 1) E_{t+1}^{ij},

and the Coulomb integral of two Hermite Gaussians is
(2 pi^(5/2) / (p q sqrt(p+q))) R_{t u v}(alpha, P - Q), alpha = pq/(p+q),

    R^n_{000} = (-2 alpha)^n F_n(alpha |P - Q|^2),
    R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_PQ R^{n+1}_{t,u,v}   (u, v likewise),

so that (ab|cd) = 2 pi^(5/2)/(p q sqrt(p+q)) sum_{tuv} E^{ab}_{tuv}
sum_{t'u'v'} (-1)^(t'+u'+v') E^{cd}_{t'u'v'} R_{t+t', u+u', v+v'}.  The Boys
function F_n(T) = int_0^1 u^(2n) exp(-T u^2) du is evaluated through the
regularised incomplete gamma function, F_n(T) = Gamma(n+1/2) P(n+1/2, T) /
(2 T^(n+1/2)), with its Taylor series below T = 1e-8.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import gamma, gammainc

from .eri import pair_list

# Cartesian components of each shell, in basis order
CART = {0: [(0, 0, 0)],
        1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
        2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]}


@dataclasses.dataclass
class ShellBasis:
    """Per basis function: centre, Cartesian exponents, and its primitives."""
    xyz: np.ndarray      # [nbf, 3]
    lmn: np.ndarray      # [nbf, 3] int
    start: np.ndarray    # [nbf + 1] int: primitives of f are [start[f], start[f+1])
    exps: np.ndarray     # [nprim]
    coefs: np.ndarray    # [nprim], the whole function's normalisation included
    atom: np.ndarray     # [nbf] int

    @property
    def nbf(self) -> int:
        return int(self.lmn.shape[0])


def double_factorial(n: int) -> int:
    return 1 if n <= 0 else n * double_factorial(n - 2)


def primitive_self_overlap(a: float, lmn) -> float:
    """int (x^l y^m z^n)^2 exp(-2 a r^2) d^3r: prod over axes of
    (2k-1)!! / (4a)^k sqrt(pi / (2a)) for each exponent k."""
    out = 1.0
    for k in lmn:
        out *= double_factorial(2 * k - 1) / (4.0 * a) ** k * math.sqrt(math.pi / (2.0 * a))
    return out


def boys(n: int, T):
    """F_n(T) = int_0^1 u^(2n) exp(-T u^2) du (array T)."""
    T = np.asarray(T, dtype=np.float64)
    small = T < 1e-8
    Ts = np.where(small, 1.0, T)
    big = gamma(n + 0.5) * gammainc(n + 0.5, Ts) / (2.0 * Ts ** (n + 0.5))
    ser = 1.0 / (2 * n + 1) - T / (2 * n + 3)
    return np.where(small, ser, big)


def hermite_e(i: int, j: int, a: float, b: float, A: float, B: float) -> np.ndarray:
    """E_t^{ij} for t = 0 .. i + j (1-D), by the recurrences above."""
    p = a + b
    P = (a * A + b * B) / p
    E = {(0, 0): np.zeros(1)}
    E[(0, 0)][0] = math.exp(-a * b / p * (A - B) ** 2)

    def get(ii, jj):
        if (ii, jj) in E:
            return E[(ii, jj)]
        if ii > 0:
            prev = get(ii - 1, jj)
            X = P - A
        else:
            prev = get(ii, jj - 1)
            X = P - B
        out = np.zeros(ii + jj + 1)
        for t in range(ii + jj + 1):
            v = 0.0
            if t - 1 >= 0 and t - 1 < len(prev):
                v += prev[t - 1] / (2.0 * p)
            if t < len(prev):
                v += X * prev[t]
            if t + 1 < len(prev):
                v += (t + 1) * prev[t + 1]
            out[t] = v
        E[(ii, jj)] = out
        return out

    return get(i, j)


def hermite_r(L: int, alpha: float, PQ) -> np.ndarray:
    """R_{tuv} = R^0_{tuv}(alpha, PQ) for t + u + v <= L, as an array [L+1]^3."""
    X, Y, Z = PQ
    T = alpha * (X * X + Y * Y + Z * Z)
    # R^n_{tuv} for n = 0..L, built from n = L down to 0
    Rn = {}
    for n in range(L + 1):
        Rn[(n, 0, 0, 0)] = (-2.0 * alpha) ** n * float(boys(n, T))

    def r(n, t, u, v):
        key = (n, t, u, v)
        if key in Rn:
            return Rn[key]
        if t < 0 or u < 0 or v < 0:
            return 0.0
        if t > 0:
            val = (t - 1) * r(n + 1, t - 2, u, v) + X * r(n + 1, t - 1, u, v)
        elif u > 0:
            val = (u - 1) * r(n + 1, t, u - 2, v) + Y * r(n + 1, t, u - 1, v)
        else:
            val = (v - 1) * r(n + 1, t, u, v - 2) + Z * r(n + 1, t, u, v - 1)
        Rn[key] = val
        return val

    out = np.zeros((L + 1, L + 1, L + 1))
    for t in range(L + 1):
        for u in range(L + 1 - t):
            for v in range(L + 1 - t - u):
                out[t, u, v] = r(0, t, u, v)
    return out


def _pair_e(a, b, A, B, la, lb):
    """E^{ab}_{tuv} = E_t^x E_u^y E_v^z as a 3-D array."""
    ex = hermite_e(la[0], lb[0], a, b, A[0], B[0])
    ey = hermite_e(la[1], lb[1], a, b, A[1], B[1])
    ez = hermite_e(la[2], lb[2], a, b, A[2], B[2])
    return ex[:, None, None] * ey[None, :, None] * ez[None, None, :]


def primitive_eri(a, A, la, b, B, lb, c, C, lc, d, D, ld) -> float:
    """(ab|cd) over unnormalised primitives x_A^l.. exp(-a |r-A|^2)."""
    p, q = a + b, c + d
    P = (a * np.asarray(A) + b * np.asarray(B)) / p
    Q = (c * np.asarray(C) + d * np.asarray(D)) / q
    Eab = _pair_e(a, b, A, B, la, lb)
    Ecd = _pair_e(c, d, C, D, lc, ld)
    L = sum(la) + sum(lb) + sum(lc) + sum(ld)
    R = hermite_r(L, p * q / (p + q), P - Q)
    tot = 0.0
    for t in range(Eab.shape[0]):
        for u in range(Eab.shape[1]):
            for v in range(Eab.shape[2]):
                if Eab[t, u, v] == 0.0:
                    continue
                for t2 in range(Ecd.shape[0]):
                    for u2 in range(Ecd.shape[1]):
                        for v2 in range(Ecd.shape[2]):
                            sgn = -1.0 if (t2 + u2 + v2) % 2 else 1.0
                            tot += Eab[t, u, v] * sgn * Ecd[t2, u2, v2] * R[t + t2, u + u2, v + v2]
    return 2.0 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * tot


def eri(basis: ShellBasis, mu: int, nu: int, lam: int, sig: int) -> float:
    """(mu nu|lam sig) over the contracted basis functions (Eq. integral)."""
    b = basis
    tot = 0.0
    for i in range(b.start[mu], b.start[mu + 1]):
        for j in range(b.start[nu], b.start[nu + 1]):
            for k in range(b.start[lam], b.start[lam + 1]):
                for m in range(b.start[sig], b.start[sig + 1]):
                    tot += (b.coefs[i] * b.coefs[j] * b.coefs[k] * b.coefs[m] *
                            primitive_eri(b.exps[i], b.xyz[mu], b.lmn[mu],
                                          b.exps[j], b.xyz[nu], b.lmn[nu],
                                          b.exps[k], b.xyz[lam], b.lmn[lam],
                                          b.exps[m], b.xyz[sig], b.lmn[sig]))
    return tot


def overlap(basis: ShellBasis, mu: int, nu: int) -> float:
    """<mu|nu> = sum of E_0^x E_0^y E_0^z (pi/p)^(3/2) over primitive pairs."""
    b = basis
    tot = 0.0
    for i in range(b.start[mu], b.start[mu + 1]):
        for j in range(b.start[nu], b.start[nu + 1]):
            a, c = b.exps[i], b.exps[j]
            e = _pair_e(a, c, b.xyz[mu], b.xyz[nu], b.lmn[mu], b.lmn[nu])
            tot += b.coefs[i] * b.coefs[j] * e[0, 0, 0] * (math.pi / (a + c)) ** 1.5
    return tot


class ShellPairs:
    """The product densities rho_I = chi_mu chi_nu, mu <= nu, of a shell basis,
    in the packed order of the s-type pairs (I = nu(nu+1)/2 + mu); the
    interface the decomposition of oracle.cd reads (npair, mu, nu)."""

    def __init__(self, basis: ShellBasis):
        self.basis = basis
        self.nbf = basis.nbf
        self.mu, self.nu = pair_list(self.nbf)

    @property
    def npair(self) -> int:
        return int(self.mu.shape[0])

    def value(self, I: int, J: int) -> float:
        return eri(self.basis, int(self.mu[I]), int(self.nu[I]), int(self.mu[J]), int(self.nu[J]))

    def column(self, J: int) -> np.ndarray:
        return np.array([self.value(I, J) for I in range(self.npair)])

    def diagonal(self) -> np.ndarray:
        return np.array([self.value(I, I) for I in range(self.npair)])

    def matrix(self) -> np.ndarray:
        n = self.npair
        V = np.empty((n, n))
        for I in range(n):
            for J in range(I, n):
                V[I, J] = V[J, I] = self.value(I, J)
        return V
