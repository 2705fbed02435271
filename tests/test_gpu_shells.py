"""The decomposition over contracted Cartesian shells (s, p, d) on the GPU
(cds_cd_decompose_shells: FP64 McMurchie-Davidson integrals, the s-type
pivot rule) against the oracle's contracted-shell integrals (pinned by
centre derivatives of the closed-form s-integrals, 8-fold symmetry and
positive semidefiniteness in tests/test_oracle_shells.py) and the oracle's
decomposition on them:

* delta = 0: L^T L reproduces the oracle's supermatrix to 1e-11 (so every
  integral the GPU made is the oracle's);
* delta in {1e-4, 1e-6}, full and atomic pivot sets: the oracle's pivot
  sequence, vectors and residuals within 1e-11;
* a larger basis (6 centres, 66 functions): the strict bound
  |V_IJ - L_I.L_J| <= delta on sampled pairs with V from the oracle, and no
  residual below -1e-12.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cd, shells

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_1459_gb300 import cdsigma as C  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu(sh, delta, scheme="full", max_rank=None):
    L, piv, D, de = C.cds_cd_decompose_shells(dev(sh.xyz), dev(sh.lmn.astype(np.int32)),
                                              dev(sh.start.astype(np.int32)), dev(sh.exps),
                                              dev(sh.coefs), dev(sh.atom.astype(np.int32)), delta,
                                              scheme, max_rank=max_rank)
    torch.cuda.synchronize()
    return L.cpu().numpy(), piv.cpu().numpy().astype(np.int64), D.cpu().numpy(), de


@pytest.fixture(scope="module")
def small():
    sh = W.shell_config(ncentre=2, seed=3)
    b = shells.ShellBasis(sh.xyz, sh.lmn, sh.start, sh.exps, sh.coefs, sh.atom)
    sp = shells.ShellPairs(b)
    return sh, sp, sp.matrix()


def test_exact_reconstruction_reproduces_oracle_integrals(small):
    sh, sp, V = small
    L, piv, D, de = gpu(sh, 0.0, max_rank=sp.npair)
    assert np.abs(L.T @ L - V).max() <= 1e-11 * np.abs(V).max()


@pytest.mark.parametrize("delta,scheme", [(1e-4, "full"), (1e-6, "full"), (1e-4, "atomic")])
def test_shell_decomposition_matches_oracle(small, delta, scheme):
    sh, sp, V = small
    ref = cd.decompose(sp, delta, scheme=scheme, atom=sh.atom, column=lambda P: V[:, P],
                       diagonal=np.diag(V))
    L, piv, D, de = gpu(sh, delta, scheme)
    assert de == pytest.approx(ref.delta_eff, rel=1e-14)
    assert np.array_equal(piv, ref.piv)
    np.testing.assert_allclose(L, ref.L, rtol=0, atol=1e-11)
    np.testing.assert_allclose(D, ref.D, rtol=0, atol=1e-11)


def test_strict_bound_on_a_larger_shell_basis():
    sh = W.shell_config(ncentre=6, seed=7)
    b = shells.ShellBasis(sh.xyz, sh.lmn, sh.start, sh.exps, sh.coefs, sh.atom)
    sp = shells.ShellPairs(b)
    delta = 1e-5
    L, piv, D, de = gpu(sh, delta)
    assert D.max() <= delta and D.min() >= -1e-12
    rng = np.random.default_rng(5)
    I = np.concatenate([rng.integers(0, sp.npair, 150), piv[:50]])
    J = np.concatenate([rng.integers(0, sp.npair, 150), piv[::-1][:50]])
    V = np.array([sp.value(int(i), int(j)) for i, j in zip(I, J)])
    approx = (L[:, I] * L[:, J]).sum(0)
    assert np.abs(V - approx).max() <= delta
