"""The hand-written adjoint (cds_qp_gradient, cds_cd_to_mo_backward) behind
torch.autograd.Function against the oracle's implicit derivative (itself
pinned by finite differences) and against central finite differences of the
GPU's own FP64 Newton roots.  Bar: relative error <= 1e-6 (FP64) and <= 1e-3
for the tensor-core form (BF16X3 / TF32X3 split GEMMs, FP32 accumulation)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import grad as ograd
from tests import oracle_pipeline as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_0912_1459_gb300 import cdsigma as C  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def close(a, b, rel):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() <= rel * max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("grad_prec,tol", [("fp64", 1e-6), ("bf16x3", 1e-3), ("tf32x3", 1e-3)])
@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_adjoint_matches_oracle_gradient(name, delta, grad_prec, tol):
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    rov, rp = O.factors(name, ref.L)
    orbs = m.orbitals[:2] if name == "c1" else m.orbitals
    rp = rp[:len(orbs)]
    eps = dev(m.eps).requires_grad_()
    Lov = dev(rov).requires_grad_()
    Lp = dev(rp).requires_grad_()
    w, st = C.QPEnergies.apply(eps, Lov, Lp, dev(orbs.astype(np.int32)), m.nocc, 1e-12, 100,
                               "fp64", False, grad_prec)
    assert torch.all(st == 0)
    gw = torch.arange(1, len(orbs) + 1, dtype=torch.float64, device=DEV)   # l = sum_t (t+1) w_t
    (w * gw).sum().backward()
    r_eps = np.zeros(m.nbf)
    r_ov = np.zeros_like(rov)
    r_p = np.zeros_like(rp)
    for t, q in enumerate(orbs):
        de, dq, dov, P = ograd.qp_gradient(rp[t], rov, m.eps, m.nocc, int(q), float(w[t].detach()))
        r_eps += (t + 1) * de
        r_ov += (t + 1) * dov
        r_p[t] += (t + 1) * dq
    assert close(eps.grad.cpu().numpy(), r_eps, tol)
    assert close(Lov.grad.cpu().numpy(), r_ov, tol)
    assert close(Lp.grad.cpu().numpy(), r_p, tol)


def test_adjoint_matches_finite_differences_and_chains_to_C():
    m = O.molecule("c0")
    ref = O.decomposition("c0", 1e-6)
    orbs = dev(m.orbitals.astype(np.int32))
    L = dev(ref.L)
    Cm = dev(m.C).requires_grad_()
    eps = dev(m.eps).requires_grad_()
    Lov, Lp = C.MOFactors.apply(Cm, L, m.nocc, orbs)
    w, st = C.QPEnergies.apply(eps, Lov, Lp, orbs, m.nocc)
    w[1].backward()        # the LUMO quasiparticle energy
    h = 1e-5

    def root(eps_, C_):
        lov, lp = C.cds_cd_to_mo(L, C_, m.nocc, orbs)
        ww, _, _, s_ = C.cds_qp_solve(lov, lp, orbs, eps_, m.nocc, conv=1e-13, max_iter=100)
        return float(ww[1])
    e0, c0 = eps.detach(), Cm.detach()
    for k in (0, 3, int(m.orbitals[1]), m.nbf - 2):
        ep, em = e0.clone(), e0.clone()
        ep[k] += h
        em[k] -= h
        fd = (root(ep, c0) - root(em, c0)) / (2 * h)
        assert abs(fd - float(eps.grad[k])) <= 1e-6 * max(1.0, abs(float(eps.grad[k])))
    rng = np.random.default_rng(2)
    for _ in range(4):
        mu, p = int(rng.integers(m.nbf)), int(rng.integers(m.nbf))
        cp, cm = c0.clone(), c0.clone()
        cp[mu, p] += h
        cm[mu, p] -= h
        fd = (root(e0, cp) - root(e0, cm)) / (2 * h)
        assert abs(fd - float(Cm.grad[mu, p])) <= 1e-6 * max(1.0, abs(float(Cm.grad[mu, p])))


@pytest.mark.parametrize("grad_prec", ["bf16x3", "tf32x3"])
def test_tensor_core_adjoint_chunks_and_ragged_shapes(grad_prec):
    """More orbitals than one chunk of the tensor-core form (8), and a single
    occupied orbital: equal to the FP64 adjoint within 1e-3 of each output's
    largest entry."""
    m = O.molecule("c1")
    ref = O.decomposition("c1", 1e-4)
    orbs = np.arange(m.nocc - 6, m.nocc + 5, dtype=np.int32)          # 11 orbitals
    rov, rp = O.factors("c1", ref.L, orbs)
    Lov, Lp, eps, o = dev(rov), dev(rp), dev(m.eps), dev(orbs)
    w, P, it, st, _ = C.cds_qp_solve_bracketed(Lov, Lp, o, eps, m.nocc, conv=1e-12)
    g = torch.linspace(-1.0, 2.0, len(orbs), dtype=torch.float64, device=DEV)
    ref_g = C.cds_qp_gradient(Lov, Lp, o, eps, m.nocc, w, g, "fp64")
    got = C.cds_qp_gradient(Lov, Lp, o, eps, m.nocc, w, g, grad_prec)
    for a, b in zip(got, ref_g):
        assert close(a.cpu().numpy(), b.cpu().numpy(), 1e-3)
    # one occupied orbital: every tile of the occupied side ragged
    o1 = torch.tensor([0, 1, 2], dtype=torch.int32, device=DEV)
    from oracle import ao2mo
    lov1, lp1 = ao2mo.mo_factors(ref.L, m.C, 1, np.array([0, 1, 2]))
    Lov1, Lp1 = dev(lov1), dev(lp1)
    w1, _, _, _, _ = C.cds_qp_solve_bracketed(Lov1, Lp1, o1, eps, 1, conv=1e-12)
    g1 = torch.ones(3, dtype=torch.float64, device=DEV)
    r1 = C.cds_qp_gradient(Lov1, Lp1, o1, eps, 1, w1, g1, "fp64")
    t1 = C.cds_qp_gradient(Lov1, Lp1, o1, eps, 1, w1, g1, grad_prec)
    for a, b in zip(t1, r1):
        assert close(a.cpu().numpy(), b.cpu().numpy(), 1e-3)
