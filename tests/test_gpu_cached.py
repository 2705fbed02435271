"""Newton from cached numerators (cds_sigma2_diag_cache + cds_qp_solve_cached)
against the recomputing path and the FP64 oracle.

* the self-energy the caching call returns is the recomputing call's, bit for
  bit (the cache store does not touch the sums);
* for quasiparticle poles (P >= 0.5) the cached Newton iteration reaches the
  recomputing one's roots within 1e-7 Ha (only the order of the FP32 partial
  sums differs), with the same status, and the iteration count within one;
* quasiparticle energies (P >= 0.5) within 0.1 meV of the FP64 oracle.
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


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "tf32x3"])
@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_cached_newton_matches_recompute_and_oracle(name, delta, prec):
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    Lov, Lp = O.factors(name, ref.L)
    rov, rp = dev(Lov), dev(Lp)
    eps, orbs = dev(m.eps), dev(m.orbitals)
    import workloads as W
    E = dev(W.energy_grid(m.eps[m.orbitals], 16))
    s0, d0 = G.cds_sigma2_diag(rov, rp, eps, m.nocc, E, prec)
    s1, d1, cache = G.cds_sigma2_diag_cache(rov, rp, eps, m.nocc, E, prec)
    # energies past the first come from the cached numerators (FP32 sums in
    # another order): equal to the single tensor-core pass up to that order
    assert torch.equal(s0[:, 0], s1[:, 0]) and torch.equal(d0[:, 0], d1[:, 0])
    torch.testing.assert_close(s1, s0, rtol=1e-5, atol=1e-9)
    torch.testing.assert_close(d1, d0, rtol=1e-5, atol=1e-8)
    w0, P0, it0, st0 = G.cds_qp_solve(rov, rp, orbs, eps, m.nocc, precision=prec)
    w1, P1, it1, st1 = G.cds_qp_solve_cached(cache, orbs, eps, m.nbf, m.nocc)
    # quasiparticle poles; a satellite's Newton path near a pole of Sigma may
    # pick another root when the sums differ in the last bits
    qp = ((st0 == 0) & (P0 >= 0.5)).cpu().numpy()
    assert qp.sum() >= 1
    assert np.array_equal(st1.cpu().numpy()[qp], st0.cpu().numpy()[qp])
    assert np.abs((it0 - it1).cpu().numpy()[qp]).max() <= 1
    assert np.abs((w0 - w1).cpu().numpy()[qp]).max() <= 1e-7
    assert np.abs((P0 - P1).cpu().numpy()[qp]).max() <= 1e-6
    res = O.solve(name, Lov, Lp, m.orbitals)
    for t, (w, P, it, st) in enumerate(res):
        if st == 0 and P >= 0.5:
            assert abs(float(w1[t]) - w) <= TOL_QP


def test_cache_too_small_is_rejected():
    m = O.molecule("c0")
    ref = O.decomposition("c0", 1e-6)
    Lov, Lp = O.factors("c0", ref.L)
    small = torch.empty(16, dtype=torch.uint8, device=DEV)
    with pytest.raises(G.CdsError):
        G.cds_qp_solve_cached(small, dev(m.orbitals), dev(m.eps), m.nbf, m.nocc)


@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_bracketed_newton_against_oracle(name, delta):
    """Safeguarded Newton (cds_qp_solve_bracketed_cached, BF16X3 numerators)
    against the oracle's bracketed solve on the same factors: every orbital
    converges, inside the oracle's pole-free interval, within 0.1 meV of the
    oracle's root, with the same pole strength to 1e-4."""
    from oracle import qp, sigma2
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    Lov, Lp = O.factors(name, ref.L)
    eps, orbs = dev(m.eps), dev(m.orbitals)
    import workloads as W
    E = dev(W.energy_grid(m.eps[m.orbitals], 4))
    _, _, cache = G.cds_sigma2_diag_cache(dev(Lov), dev(Lp), eps, m.nocc, E, "bf16x3")
    w, P, it, st, br = G.cds_qp_solve_bracketed_cached(cache, orbs, eps, m.nbf, m.nocc)
    w, P, st, br = w.cpu().numpy(), P.cpu().numpy(), st.cpu().numpy(), br.cpu().numpy()
    for t, q in enumerate(m.orbitals):
        lo, hi = qp.pole_bracket(m.eps, m.nocc, m.eps[q])

        def f(x, t=t):
            a, d = sigma2.sigma2_from_factors(Lp[t], Lov, m.eps, m.nocc, [x])
            return a[0], d[0]
        wr, Pr, itr, str_ = qp.bracketed_qp(f, m.eps[q], lo, hi)
        assert st[t] == 0 and str_ == 0
        assert lo < w[t] < hi and br[t, 0] <= w[t] <= br[t, 1]
        assert abs(w[t] - wr) <= TOL_QP
        assert abs(P[t] - Pr) <= 1e-4 * abs(Pr)


@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_grid_from_cached_numerators(name, delta):
    """With the numerators kept, the tensor-core epilogue evaluates the first
    energy of each orbital and the cached-numerator kernel the other 63: the
    same sums as the single tensor-core pass up to FP32 summation order
    (within 1e-5 relative; the first energy identical), and within the
    split-precision bar of the FP64 path."""
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    Lov, Lp = O.factors(name, ref.L)
    rov, rp = dev(Lov), dev(Lp)
    eps = dev(m.eps)
    import workloads as W
    E = dev(W.energy_grid(m.eps[m.orbitals], 64))
    s0, d0 = G.cds_sigma2_diag(rov, rp, eps, m.nocc, E, "bf16x3")
    s1, d1, _ = G.cds_sigma2_diag_cache(rov, rp, eps, m.nocc, E, "bf16x3")
    assert torch.equal(s0[:, 0], s1[:, 0]) and torch.equal(d0[:, 0], d1[:, 0])
    torch.testing.assert_close(s1, s0, rtol=1e-5, atol=1e-9)
    torch.testing.assert_close(d1, d0, rtol=1e-5, atol=1e-8)
    s64, _ = G.cds_sigma2_diag(rov, rp, eps, m.nocc, E, "fp64")
    assert (s1 - s64).abs().max().item() <= 3.67e-6 + 1e-5 * s64.abs().max().item()


@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_fp64_cached_newton_equals_recomputing_fp64(name, delta):
    """FP64 numerator cache: the grid pass equals cds_sigma2_diag (FP64) bit
    for bit, and Newton from the cache (plain and safeguarded) reaches the
    recomputing FP64 solvers' roots exactly (same per-element arithmetic and
    order of sums at every energy), i.e. the oracle's within 1e-10 Ha."""
    import workloads as W
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    Lov, Lp = O.factors(name, ref.L)
    rov, rp, eps, orbs = dev(Lov), dev(Lp), dev(m.eps), dev(m.orbitals)
    E = dev(W.energy_grid(m.eps[m.orbitals], 8))
    s0, d0 = G.cds_sigma2_diag(rov, rp, eps, m.nocc, E, "fp64")
    s1, d1, cache = G.cds_sigma2_diag_cache(rov, rp, eps, m.nocc, E, "fp64")
    assert torch.equal(s0, s1) and torch.equal(d0, d1)
    w0, P0, it0, st0 = G.cds_qp_solve(rov, rp, orbs, eps, m.nocc, conv=1e-10, precision="fp64")
    w1, P1, it1, st1 = G.cds_qp_solve_cached(cache, orbs, eps, m.nbf, m.nocc, conv=1e-10,
                                             precision="fp64")
    assert torch.equal(w0, w1) and torch.equal(P0, P1) and torch.equal(it0, it1)
    assert torch.equal(st0, st1)
    b0 = G.cds_qp_solve_bracketed(rov, rp, orbs, eps, m.nocc, conv=1e-10, precision="fp64")
    b1 = G.cds_qp_solve_bracketed_cached(cache, orbs, eps, m.nbf, m.nocc, conv=1e-10,
                                         precision="fp64")
    for a, b in zip(b0, b1):
        assert torch.equal(a, b)
    res = O.solve(name, Lov, Lp, m.orbitals, conv=1e-10)
    for t, (w, P, it, st) in enumerate(res):
        if st == 0:
            assert abs(float(w1[t]) - w) <= 1e-10
