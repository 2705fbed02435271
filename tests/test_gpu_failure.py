"""Device-side failure reporting and the recomputing safeguarded Newton.

* The bounded wait of the tensor-core kernels: run on an mbarrier phase that
  nothing completes (a flag nobody sets), it gives up after its limit, leaves
  CDS_ERR_TIMEOUT in the error word, and the kernel returns -- the context
  stays usable (a decomposition right after it matches the oracle).
* Newton that runs out of iterations (max_iter = 1) reports
  CDS_ERR_NO_CONVERGENCE from the call and CDS_QP_NO_CONVERGENCE per orbital,
  with the outputs of its one step written.
* cds_qp_solve_bracketed (Sigma recomputed every iteration, FP64 or BF16X3)
  against the oracle's bracketed solve: every orbital converges inside the
  oracle's pole-free interval; FP64 within 1e-10 Ha of the oracle's root,
  BF16X3 within 0.1 meV.
"""
import numpy as np
import pytest
import torch

import oracle_pipeline as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0912_1459_gb300 as G  # noqa: E402

DEV = torch.device("cuda:0")
TOL_QP = 0.1e-3 / 27.211396


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_bounded_wait_gives_up_and_context_survives():
    for seconds in (0.01, 0.05):
        assert G.cds_wait_check(seconds) == 8          # CDS_ERR_TIMEOUT, no hang, no trap
    # the context still works: a decomposition right after matches the oracle's pivots
    m = O.molecule("c0")
    ref = O.decomposition("c0", m.delta)
    L, piv, D, _ = G.cds_cd_decompose(dev(m.basis.xyz), dev(m.basis.alpha),
                                      dev(m.basis.atom.astype(np.int32)), m.delta, "full")
    torch.cuda.synchronize()
    assert np.array_equal(piv.cpu().numpy(), ref.piv)
    assert G.cds_wait_check(3.0) == 1                  # limits outside (0, 2] s: CDS_ERR_ARG


def test_newton_out_of_iterations_reports_status():
    m = O.molecule("c0")
    ref = O.decomposition("c0", m.delta)
    Lov, Lp = O.factors("c0", ref.L)
    orbs = dev(m.orbitals)
    with pytest.raises(G.CdsError) as ei:
        G.cds_qp_solve(dev(Lov), dev(Lp), orbs, dev(m.eps), m.nocc, max_iter=1,
                       raise_on_nonconvergence=True)
    assert ei.value.status == 5
    w, P, it, st = G.cds_qp_solve(dev(Lov), dev(Lp), orbs, dev(m.eps), m.nocc, max_iter=1)
    assert np.all(st.cpu().numpy() == 1) and np.all(it.cpu().numpy() == 1)
    # the one step taken is the oracle's first Newton step
    from oracle import sigma2
    for t, q in enumerate(m.orbitals):
        s, d = sigma2.sigma2_from_factors(Lp[t], Lov, m.eps, m.nocc, [m.eps[q]])
        Pr = 1.0 / (1.0 - d[0])
        wr = m.eps[q] + s[0] * Pr
        assert abs(float(w[t]) - wr) <= 1e-10 and abs(float(P[t]) - Pr) <= 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x3", TOL_QP)])
@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_bracketed_newton_recomputing_against_oracle(name, delta, prec, tol):
    from oracle import qp, sigma2
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    Lov, Lp = O.factors(name, ref.L)
    w, P, it, st, br = G.cds_qp_solve_bracketed(dev(Lov), dev(Lp), dev(m.orbitals), dev(m.eps),
                                                m.nocc, conv=1e-10, precision=prec)
    w, P, st, br = w.cpu().numpy(), P.cpu().numpy(), st.cpu().numpy(), br.cpu().numpy()
    for t, q in enumerate(m.orbitals):
        lo, hi = qp.pole_bracket(m.eps, m.nocc, m.eps[q])

        def f(x, t=t):
            a, d = sigma2.sigma2_from_factors(Lp[t], Lov, m.eps, m.nocc, [x])
            return a[0], d[0]
        wr, Pr, itr, str_ = qp.bracketed_qp(f, m.eps[q], lo, hi, conv=1e-10)
        assert st[t] == 0 and str_ == 0
        assert lo < w[t] < hi and br[t, 0] <= w[t] <= br[t, 1]
        assert abs(w[t] - wr) <= tol
        assert abs(P[t] - Pr) <= (1e-8 if prec == "fp64" else 1e-4) * abs(Pr)
