"""Test helper: the whole method run through the CPU oracle, cached per case."""
import functools

import numpy as np

import workloads as W
from oracle import ao2mo, cd, eri, qp, sigma2


@functools.lru_cache(maxsize=None)
def molecule(name: str):
    return {"c0": W.config0, "c1": W.config1, "c2": W.config2}[name]()


@functools.lru_cache(maxsize=None)
def pairs(name: str):
    m = molecule(name)
    return eri.PairData(m.basis.xyz, m.basis.alpha)


@functools.lru_cache(maxsize=None)
def decomposition(name: str, delta: float, scheme: str = "full"):
    m = molecule(name)
    return cd.decompose(pairs(name), delta, scheme=scheme, atom=m.basis.atom)


def factors(name: str, L: np.ndarray, orbitals=None):
    m = molecule(name)
    orbs = m.orbitals if orbitals is None else np.asarray(orbitals)
    return ao2mo.mo_factors(L, m.C, m.nocc, orbs)


def sigma(name: str, Lov, Lp, E):
    """[np, nE] Sigma and dSigma for every row of Lp."""
    m = molecule(name)
    out = [sigma2.sigma2_from_factors(Lp[t], Lov, m.eps, m.nocc, E[t]) for t in range(Lp.shape[0])]
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


def solve(name: str, Lov, Lp, orbitals, conv=1e-5, max_iter=50):
    m = molecule(name)
    res = []
    for t, q in enumerate(orbitals):
        def f(w, t=t):
            s, d = sigma2.sigma2_from_factors(Lp[t], Lov, m.eps, m.nocc, [w])
            return s[0], d[0]
        res.append(qp.newton_qp(f, m.eps[q], conv=conv, max_iter=max_iter))
    return res
