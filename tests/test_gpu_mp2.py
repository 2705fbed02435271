"""MP2 correlation energy (Eq. MP2) on the GPU against the oracle.

The oracle's Eq. MP2 from the factors is pinned in test_oracle_ao2mo_sigma.py
(explicit-integral loop, per-i split into the 2p1h self-energy, o = v = 1
closed form).  Here the same factors go through cds_mp2_energy:
* FP64 path: per-i sums within 1e-12 relative of the largest |e_i| (tiny case)
  and 1e-11 (ring case);
* split precisions: total within 1e-5 relative (+1e-7 Ha) of the FP64 oracle,
  the bound the self-energy's split path meets;
* edge cases: no virtual orbitals, rank 0.
"""
import numpy as np
import pytest
import torch

import oracle_pipeline as O
from oracle import sigma2

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0912_1459_gb300 as G  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def oracle_factors(name, delta):
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    Lov, Lp = O.factors(name, ref.L)
    return m, Lov


@pytest.mark.parametrize("name,delta,tol", [("c0", 1e-6, 1e-12), ("c1", 1e-4, 1e-11)])
def test_mp2_fp64_parity(name, delta, tol):
    m, Lov = oracle_factors(name, delta)
    ref_i = sigma2.mp2_from_factors(Lov, m.eps, m.nocc, pairs=True)
    tot, e_i = G.cds_mp2_energy(dev(Lov), dev(m.eps), m.nocc, "fp64")
    e_i = e_i.cpu().numpy()
    np.testing.assert_allclose(e_i, ref_i, rtol=0, atol=tol * np.abs(ref_i).max())
    assert float(tot) == pytest.approx(ref_i.sum(), rel=tol)
    assert float(tot) < 0


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-4)])
def test_mp2_split_precision(name, delta, prec):
    m, Lov = oracle_factors(name, delta)
    ref = sigma2.mp2_from_factors(Lov, m.eps, m.nocc)
    tot, e_i = G.cds_mp2_energy(dev(Lov), dev(m.eps), m.nocc, prec)
    assert abs(float(tot) - ref) <= 1e-5 * abs(ref) + 1e-7
    assert float(e_i.sum()) == pytest.approx(float(tot), rel=1e-13)


def test_mp2_edge_cases():
    m, Lov = oracle_factors("c0", 1e-6)
    # rank 0: every integral is zero
    L0 = torch.zeros((m.nocc, m.nbf - m.nocc, 0), dtype=torch.float64, device=DEV)
    for prec in ("fp64", "bf16x3"):
        tot, e_i = G.cds_mp2_energy(L0, dev(m.eps), m.nocc, prec)
        assert float(tot) == 0.0 and torch.all(e_i == 0)
    # a single occupied orbital: the i = j terms only
    tot, e_i = G.cds_mp2_energy(dev(Lov[:1]), dev(m.eps[:1].tolist() + m.eps[m.nocc:].tolist()),
                                1, "fp64")
    ref = sigma2.mp2_from_factors(Lov[:1], np.concatenate([m.eps[:1], m.eps[m.nocc:]]), 1)
    assert float(tot) == pytest.approx(ref, rel=1e-12)
