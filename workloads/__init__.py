"""Seeded synthetic workloads for the Cholesky-factorised Sigma(2) propagator.

This module only *draws inputs*: Gaussian centres and exponents, MO
coefficients, orbital energies, orbital selections and energy grids.  It holds
none of the method's arithmetic (no electron-repulsion integral, no Cholesky
step, no transform, no self-energy, no Newton step) and is shared by the CPU
oracle, the GPU tests and the benchmark.

The paper's workload is C60 with contracted cc-pVXZ basis sets (Sec. III);
neither those basis sets nor an SCF exist here, so every input is a seeded
stand-in of the same shape:

* basis: normalised s-type primitive Gaussians, ``g(r) = (2a/pi)^(3/4)
  exp(-a |r-A|^2)``, a fixed geometric exponent ladder on every centre;
* MOs: ``C = S^(-1/2) Q`` with ``Q`` a seeded random orthogonal matrix, so
  ``C^T S C = 1`` like SCF orbitals (the s-Gaussian overlap ``S`` is computed
  here only to orthonormalise ``C``; it is not part of the method);
* energies: occupied uniform in [-1.5, -0.3] Ha, virtual uniform in
  [0.05, 3] Ha, sorted ascending (Koopmans-like ordering, Sec. II.B).

Layouts (shared with the C ABI): ``xyz[nbf][3]`` in bohr, ``alpha[nbf]``,
``atom[nbf]`` (centre index of each function), ``C[nbf][nmo]`` row-major with
column ``p`` the coefficients of MO ``p``.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

__all__ = [
    "Basis", "Molecule", "config0", "config1", "config2", "config3",
    "geometric_exponents", "ring_centres", "truncated_icosahedron",
    "random_cube_centres", "ball_centres", "make_basis", "s_overlap",
    "mo_coefficients", "orbital_energies", "gap_orbitals", "energy_grid",
    "make_molecule", "npair", "ShellInput", "shell_basis", "shell_config",
]


def npair(nbf: int) -> int:
    """Number of product densities I=(mu,nu), mu<=nu (Sec. II.A)."""
    return nbf * (nbf + 1) // 2


@dataclasses.dataclass
class Basis:
    xyz: np.ndarray      # [nbf, 3] float64, bohr
    alpha: np.ndarray    # [nbf] float64
    atom: np.ndarray     # [nbf] int32, centre index
    centres: np.ndarray  # [ncentre, 3]

    @property
    def nbf(self) -> int:
        return int(self.alpha.shape[0])


@dataclasses.dataclass
class Molecule:
    name: str
    basis: Basis
    C: np.ndarray        # [nbf, nmo] float64
    eps: np.ndarray      # [nmo] float64, ascending
    nocc: int
    orbitals: np.ndarray  # [np] int32, orbitals whose Sigma/QP is wanted
    nE: int
    delta: float
    seed: int

    @property
    def nbf(self) -> int:
        return self.basis.nbf

    @property
    def nvir(self) -> int:
        return self.C.shape[1] - self.nocc


def geometric_exponents(lo: float, hi: float, n: int) -> np.ndarray:
    return lo * (hi / lo) ** (np.arange(n, dtype=np.float64) / (n - 1))


def random_cube_centres(n: int, edge: float, min_sep: float,
                        rng: np.random.Generator) -> np.ndarray:
    """Uniform points in [0, edge]^3, redrawn until all pairs are >= min_sep."""
    pts: list[np.ndarray] = []
    while len(pts) < n:
        p = rng.uniform(0.0, edge, size=3)
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts, dtype=np.float64)


def ball_centres(n: int, radius: float, min_sep: float,
                 rng: np.random.Generator) -> np.ndarray:
    """Uniform points in a ball of the given radius, pairwise >= min_sep."""
    pts: list[np.ndarray] = []
    while len(pts) < n:
        p = rng.uniform(-radius, radius, size=3)
        if np.dot(p, p) > radius * radius:
            continue
        if all(np.linalg.norm(p - q) >= min_sep for q in pts):
            pts.append(p)
    return np.array(pts, dtype=np.float64)


def ring_centres(n: int, radius: float) -> np.ndarray:
    t = 2.0 * math.pi * np.arange(n) / n
    return np.stack([radius * np.cos(t), radius * np.sin(t), np.zeros(n)], axis=1)


def truncated_icosahedron(edge: float) -> np.ndarray:
    """The 60 vertices of a truncated icosahedron (C60 cage) with the given edge.

    Cyclic (even) permutations of (0, +-1, +-3phi), (+-1, +-(2+phi), +-2phi)
    and (+-phi, +-2, +-(2phi+1)) give edge 2; the set is then scaled.
    """
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    base = [(0.0, 1.0, 3 * phi), (1.0, 2 + phi, 2 * phi), (phi, 2.0, 2 * phi + 1)]
    pts = set()
    for b in base:
        for cyc in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
            v = (b[cyc[0]], b[cyc[1]], b[cyc[2]])
            for s in itertools.product((1.0, -1.0), repeat=3):
                pts.add(tuple(round(s[k] * v[k], 12) + 0.0 for k in range(3)))
    arr = np.array(sorted(pts), dtype=np.float64)
    assert arr.shape == (60, 3)
    return arr * (edge / 2.0)


def make_basis(centres: np.ndarray, exponents: np.ndarray) -> Basis:
    """Same exponent ladder on every centre; functions ordered centre-major."""
    nc, ne = centres.shape[0], exponents.shape[0]
    xyz = np.repeat(centres, ne, axis=0).astype(np.float64)
    alpha = np.tile(exponents, nc).astype(np.float64)
    atom = np.repeat(np.arange(nc, dtype=np.int32), ne)
    return Basis(xyz=np.ascontiguousarray(xyz), alpha=alpha, atom=atom,
                 centres=centres.astype(np.float64))


def s_overlap(basis: Basis) -> np.ndarray:
    """Overlap of normalised s-Gaussians (input generation only):
    S_mn = (2 sqrt(a_m a_n)/(a_m+a_n))^(3/2) exp(-a_m a_n/(a_m+a_n) |A-B|^2)."""
    a = basis.alpha
    p = a[:, None] + a[None, :]
    r2 = ((basis.xyz[:, None, :] - basis.xyz[None, :, :]) ** 2).sum(-1)
    return (2.0 * np.sqrt(a[:, None] * a[None, :]) / p) ** 1.5 * np.exp(
        -a[:, None] * a[None, :] / p * r2)


def mo_coefficients(basis: Basis, rng: np.random.Generator) -> np.ndarray:
    """C = S^(-1/2) Q with Q from the QR of a seeded Gaussian matrix."""
    S = s_overlap(basis)
    w, U = np.linalg.eigh(S)
    if w.min() <= 0:
        raise ValueError("overlap matrix not positive definite")
    s_inv_half = (U / np.sqrt(w)) @ U.T
    G = rng.standard_normal((basis.nbf, basis.nbf))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))
    return np.ascontiguousarray(s_inv_half @ Q)


def orbital_energies(nocc: int, nvir: int, rng: np.random.Generator) -> np.ndarray:
    occ = np.sort(rng.uniform(-1.5, -0.3, size=nocc))
    vir = np.sort(rng.uniform(0.05, 3.0, size=nvir))
    return np.concatenate([occ, vir]).astype(np.float64)


def gap_orbitals(nocc: int, n_below: int, n_above: int) -> np.ndarray:
    """Orbitals nocc-n_below .. nocc+n_above-1 (0-based): HOMO down, LUMO up."""
    return np.arange(nocc - n_below, nocc + n_above, dtype=np.int32)


def energy_grid(eps_q: np.ndarray, nE: int, half_width: float = 0.25) -> np.ndarray:
    """E_k = eps_q + (-w + 2w k/(nE-1)), k = 0..nE-1; shape [np, nE]."""
    eps_q = np.asarray(eps_q, dtype=np.float64)
    if nE == 1:
        return eps_q[:, None].copy()
    off = -half_width + 2.0 * half_width * np.arange(nE) / (nE - 1)
    return eps_q[:, None] + off[None, :]


def make_molecule(name: str, centres: np.ndarray, exponents: np.ndarray,
                  nocc: int, orbitals: np.ndarray, nE: int, delta: float,
                  rng: np.random.Generator, seed: int) -> Molecule:
    basis = make_basis(centres, exponents)
    C = mo_coefficients(basis, rng)
    eps = orbital_energies(nocc, basis.nbf - nocc, rng)
    return Molecule(name=name, basis=basis, C=C, eps=eps, nocc=nocc,
                    orbitals=np.asarray(orbitals, dtype=np.int32), nE=nE,
                    delta=delta, seed=seed)


def config0(seed: int = 0) -> Molecule:
    """Tiny: 6 centres uniform in a 6-bohr cube (separation >= 1 bohr), 4
    s-Gaussians each (0.1..10 geometric), N=24, o=6, delta=1e-6; HOMO and
    LUMO on 16 energy points."""
    rng = np.random.default_rng(seed)
    centres = random_cube_centres(6, 6.0, 1.0, rng)
    return make_molecule("tiny-N24", centres, geometric_exponents(0.1, 10.0, 4),
                         6, gap_orbitals(6, 1, 1), 16, 1e-6, rng, seed)


def config1(seed: int = 1) -> Molecule:
    """Mid: 20 centres on a ring of radius 8 bohr, 12 s-Gaussians each
    (0.1..10 geometric), N=240, o=40; the 10 orbitals nearest the gap."""
    rng = np.random.default_rng(seed)
    centres = ring_centres(20, 8.0)
    return make_molecule("ring-N240", centres, geometric_exponents(0.1, 10.0, 12),
                         40, gap_orbitals(40, 5, 5), 16, 1e-5, rng, seed)


def config2(seed: int = 2, delta: float = 1e-4, n_orb: int = 20, nE: int = 64) -> Molecule:
    """C60-shaped: truncated-icosahedron cage with a 2.70-bohr edge, 14
    s-Gaussians per centre (0.08..30 geometric), N=840, o=180, v=660; 20
    orbitals around the gap on 64 energy points."""
    rng = np.random.default_rng(seed)
    centres = truncated_icosahedron(2.70)
    return make_molecule("c60-N840", centres, geometric_exponents(0.08, 30.0, 14),
                         180, gap_orbitals(180, n_orb // 2, n_orb - n_orb // 2),
                         nE, delta, rng, seed)


def config3(seed: int = 3, n_clusters: int = 64) -> list[Molecule]:
    """Batched: clusters of U{4..40} centres uniform in a ball of radius
    3 n^(1/3) bohr (separation >= 1 bohr), 10 s-Gaussians each (0.1..10),
    o = N/5, delta=1e-5; each cluster has U{4..16} gap orbitals on U{8..64}
    energy points."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_clusters):
        nat = int(rng.integers(4, 41))
        centres = ball_centres(nat, 3.0 * nat ** (1.0 / 3.0), 1.0, rng)
        nbf = 10 * nat
        nocc = nbf // 5
        norb = int(rng.integers(4, 17))
        nE = int(rng.integers(8, 65))
        orbs = gap_orbitals(nocc, norb // 2, norb - norb // 2)
        out.append(make_molecule(f"cluster{c}-N{nbf}", centres,
                                 geometric_exponents(0.1, 10.0, 10), nocc, orbs,
                                 nE, 1e-5, rng, seed))
    return out


# ---------------------------------------------------------------------------
# Contracted Cartesian shells (s, p, d): seeded stand-ins for the paper's
# contracted cc-pVXZ sets (Sec. III), which are not available here.
# ---------------------------------------------------------------------------
_CART = {0: [(0, 0, 0)],
         1: [(1, 0, 0), (0, 1, 0), (0, 0, 1)],
         2: [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]}


def _dfact(n: int) -> int:
    return 1 if n <= 0 else n * _dfact(n - 2)


@dataclasses.dataclass
class ShellInput:
    """Per basis function: centre, Cartesian exponents (l, m, n), and its
    primitives [start[f], start[f+1]) with exponents and coefficients (the
    coefficients make the contracted function's self-overlap 1)."""
    xyz: np.ndarray      # [nbf, 3] float64
    lmn: np.ndarray      # [nbf, 3] int32
    start: np.ndarray    # [nbf + 1] int32
    exps: np.ndarray     # [nprim] float64
    coefs: np.ndarray    # [nprim] float64
    atom: np.ndarray     # [nbf] int32
    centres: np.ndarray

    @property
    def nbf(self) -> int:
        return int(self.lmn.shape[0])


def shell_basis(centres: np.ndarray, shells, rng: np.random.Generator) -> ShellInput:
    """shells: list of (l, exponents) per centre (the same on every centre);
    contraction coefficients drawn uniform in [0.2, 1], then scaled so that
    each Cartesian function has unit self-overlap (one-centre Gaussian
    moments: int x^2k exp(-c x^2) dx = (2k-1)!! / (2c)^k sqrt(pi / c))."""
    coefs_by_shell = [rng.uniform(0.2, 1.0, len(e)) for _, e in shells]
    xyz, lmn, start, exps, coefs, atom = [], [], [0], [], [], []
    for a, A in enumerate(np.asarray(centres, dtype=np.float64)):
        for (l, e), c in zip(shells, coefs_by_shell):
            e = np.asarray(e, dtype=np.float64)
            for comp in _CART[l]:
                S = 0.0
                for i in range(len(e)):
                    for j in range(len(e)):
                        g = e[i] + e[j]
                        m = 1.0
                        for k in comp:
                            m *= _dfact(2 * k - 1) / (2.0 * g) ** k * math.sqrt(math.pi / g)
                        S += c[i] * c[j] * m
                xyz.append(A)
                lmn.append(comp)
                exps.extend(e.tolist())
                coefs.extend((c / math.sqrt(S)).tolist())
                start.append(start[-1] + len(e))
                atom.append(a)
    return ShellInput(np.array(xyz), np.array(lmn, dtype=np.int32),
                      np.array(start, dtype=np.int32), np.array(exps), np.array(coefs),
                      np.array(atom, dtype=np.int32), np.asarray(centres, dtype=np.float64))


def shell_config(ncentre: int = 6, seed: int = 7) -> ShellInput:
    """Contracted s/p/d test basis: ncentre centres uniform in a cube of side
    2 ncentre^(1/3) + 4 bohr (separation >= 1.5), per centre a 3-primitive
    s, a 1-primitive s, a 2-primitive p and a 1-primitive d shell (11
    Cartesian functions), exponents a seeded geometric ladder."""
    rng = np.random.default_rng(seed)
    side = 2.0 * ncentre ** (1.0 / 3.0) + 4.0
    centres = random_cube_centres(ncentre, side, 1.5, rng)
    shells = [(0, geometric_exponents(0.3, 12.0, 3) * rng.uniform(0.9, 1.1)),
              (0, [0.12 * rng.uniform(0.9, 1.1)]),
              (1, geometric_exponents(0.25, 2.5, 2) * rng.uniform(0.9, 1.1)),
              (2, [0.8 * rng.uniform(0.9, 1.1)])]
    return shell_basis(centres, shells, rng)
