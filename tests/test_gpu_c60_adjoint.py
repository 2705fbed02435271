"""The adjoint at full C60 size (N = 840, o = 180, v = 660, delta = 1e-4):
quasiparticle energies of 8 orbitals around the gap differentiated with
respect to the orbital energies eps (840 values) and the MO factors Lov, Lp.

The roots are the quasiparticle solutions in the pole-free interval around
each eps_q (safeguarded Newton, FP64, converged to 1e-13 Ha).  On this
stand-in the occupied side is dense in 2h1p poles and several near-gap
occupied orbitals have no root with pole strength above 0.01 even there, so
the 8 orbitals are the ones nearest the gap (among HOMO-9 .. LUMO+9) whose
quasiparticle pole strength exceeds 0.5; finite differences with a 1e-5 step
are then meaningful.  Checks:
* FP64 adjoint against the oracle's implicit derivative on a 2-orbital subset
  (the occupied and the virtual orbital nearest the gap), relative to each
  output's largest entry: <= 1e-6;
* the tensor-core form (BF16X3 split GEMMs, FP32 accumulation) against the
  same oracle values (<= 1e-3), and BF16X3 / TF32X3 against the FP64 adjoint
  for all 8 orbitals (<= 1e-3);
* FP64 adjoint against central differences of the GPU's own FP64 roots
  (step 1e-5) for entries of eps, Lov and Lp.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import grad as ograd

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0912_1459_gb300 as G  # noqa: E402
from paper_0912_1459_gb300 import cdsigma as C  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def c60():
    m = W.config2(delta=1e-4)
    L, piv, D, de = G.cds_cd_decompose(dev(m.basis.xyz), dev(m.basis.alpha),
                                       dev(m.basis.atom.astype(np.int32)), 1e-4, "full",
                                       max_rank=2048)
    # screen HOMO-9 .. LUMO+9 with the split-precision safeguarded solve
    cand = np.arange(m.nocc - 10, m.nocc + 10, dtype=np.int32)
    Lov, Lpc = G.cds_cd_to_mo(L, dev(m.C), m.nocc, dev(cand))
    eps = dev(m.eps)
    _, Pc, _, stc, _ = G.cds_qp_solve_bracketed(Lov, Lpc, dev(cand), eps, m.nocc,
                                                precision="bf16x3")
    ok = (Pc.cpu().numpy() > 0.55) & (stc.cpu().numpy() == 0)
    near = np.argsort(np.abs(cand - (m.nocc - 0.5)), kind="stable")
    sel = np.sort([int(k) for k in near if ok[k]][:8])
    assert len(sel) == 8
    orbs = cand[sel]
    Lp = Lpc[torch.from_numpy(sel).to(DEV)].contiguous()
    o = dev(orbs)
    w, P, it, st, br = G.cds_qp_solve_bracketed(Lov, Lp, o, eps, m.nocc, conv=1e-13,
                                                precision="fp64")
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    assert np.all(P.cpu().numpy() > 0.5)
    occ = [t for t in range(8) if orbs[t] < m.nocc]
    vir = [t for t in range(8) if orbs[t] >= m.nocc]
    assert occ and vir
    sub = (occ[-1], vir[0])                                        # nearest the gap on each side
    g_sub = np.zeros(len(orbs))
    g_sub[sub[0]], g_sub[sub[1]] = 1.0, 2.0
    g_all = np.linspace(-1.0, 2.5, len(orbs))
    return m, orbs, Lov, Lp, eps, o, w, dev(g_sub), dev(g_all), sub


def test_fp64_and_tensor_core_adjoint_against_oracle_subset(c60):
    m, orbs, Lov, Lp, eps, o, w, g_sub, g_all, sub = c60
    got64 = C.cds_qp_gradient(Lov, Lp, o, eps, m.nocc, w, g_sub, "fp64")
    gotbf = C.cds_qp_gradient(Lov, Lp, o, eps, m.nocc, w, g_sub, "bf16x3")
    torch.cuda.synchronize()
    rov = Lov.cpu().numpy()
    r_eps = np.zeros(m.nbf)
    r_ov = np.zeros_like(rov)
    r_p = np.zeros(Lp.shape)
    for t, gt in ((sub[0], 1.0), (sub[1], 2.0)):
        de, dq, dov, P = ograd.qp_gradient(Lp[t].cpu().numpy(), rov, m.eps, m.nocc,
                                           int(orbs[t]), float(w[t]))
        r_eps += gt * de
        r_ov += gt * dov
        r_p[t] = gt * dq
    for name, got, tol in (("fp64", got64, 1e-6), ("bf16x3", gotbf, 1e-3)):
        e = [rel(x.cpu().numpy(), r) for x, r in zip(got, (r_eps, r_ov, r_p))]
        print(name, "rel err d_eps / d_Lov / d_Lp:", e)
        assert max(e) <= tol, (name, e)


def test_tensor_core_adjoint_all_gap_orbitals(c60):
    m, orbs, Lov, Lp, eps, o, w, g_sub, g_all, sub = c60
    ref = C.cds_qp_gradient(Lov, Lp, o, eps, m.nocc, w, g_all, "fp64")
    for prec in ("bf16x3", "tf32x3"):
        got = C.cds_qp_gradient(Lov, Lp, o, eps, m.nocc, w, g_all, prec)
        e = [rel(a.cpu().numpy(), b.cpu().numpy()) for a, b in zip(got, ref)]
        print(prec, "vs fp64 adjoint:", e)
        assert max(e) <= 1e-3, (prec, e)


def test_fp64_adjoint_against_central_differences(c60):
    m, orbs, Lov, Lp, eps, o, w, g_sub, g_all, sub = c60
    t = sub[1]                                                     # the virtual orbital
    gt = torch.zeros(len(orbs), dtype=torch.float64, device=DEV)
    gt[t] = 1.0
    d_eps, d_ov, d_p = C.cds_qp_gradient(Lov, Lp, o, eps, m.nocc, w, gt, "fp64")
    h = 1e-5
    o1 = o[t:t + 1]

    def root(eps_=eps, lov=Lov, lp=Lp[t:t + 1].contiguous()):
        ww, P, _, st, _ = G.cds_qp_solve_bracketed(lov, lp, o1, eps_, m.nocc, conv=1e-13,
                                                   precision="fp64")
        assert int(st[0]) == 0
        return float(ww[0])

    def check(fd, an):
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)

    q = int(orbs[t])
    for k in (q, m.nocc - 1, m.nocc + 7):                          # eps_q, eps_HOMO, a virtual
        ep, em = eps.clone(), eps.clone()
        ep[k] += h
        em[k] -= h
        check((root(eps_=ep) - root(eps_=em)) / (2 * h), float(d_eps[k]))
    i, a, K = m.nocc - 1, 0, 0                                     # (HOMO, LUMO) pair, first vector
    lp_, lm_ = Lov.clone(), Lov.clone()
    lp_[i, a, K] += h
    lm_[i, a, K] -= h
    check((root(lov=lp_) - root(lov=lm_)) / (2 * h), float(d_ov[i, a, K]))
    r = m.nocc + 1
    pp, pm = Lp[t:t + 1].clone(), Lp[t:t + 1].clone()
    pp[0, r, K] += h
    pm[0, r, K] -= h
    check((root(lp=pp) - root(lp=pm)) / (2 * h), float(d_p[t, r, K]))
