"""Split-precision (BF16X3 / FP16X3 / TF32X3, tcgen05) self-energy and Newton solve vs the FP64 oracle.

Bar: quasiparticle energies within 0.1 meV = 3.67e-6 Ha of the
FP64 oracle.  Sigma on the energy grid: |dSigma| <= 3.67e-6 Ha + 1e-5 |Sigma|
(the relative part covers grid points next to a pole, where the same
numerator error is amplified by the denominator).  Sizes: o = 6/40,
v = 18/200 against 128-row tiles (single ragged tile, several tiles with a
ragged tail), J = 117..472 against 32-wide k-blocks (ragged tail).
"""
import numpy as np
import pytest
import torch

import workloads as W
from tests import oracle_pipeline as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0912_1459_gb300 as G  # noqa: E402

DEV = torch.device("cuda:0")
MEV = 1e-3 / 27.211396          # 1 meV in hartree (Sec. III conversion factor)
TOL_QP = 0.1 * MEV


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "tf32x3"])
@pytest.mark.parametrize("name,delta,nE", [("c0", 1e-6, 16), ("c0", 1e-6, 1), ("c1", 1e-5, 16),
                                          ("c1", 1e-5, 5)])
def test_sigma_split_vs_oracle(name, delta, nE, prec):
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    rov, rp = O.factors(name, ref.L)
    E = W.energy_grid(m.eps[m.orbitals], nE)
    s, ds = G.cds_sigma2_diag(dev(rov), dev(rp), dev(m.eps), m.nocc, dev(E), prec)
    rs, rds = O.sigma(name, rov, rp, E)
    s = s.cpu().numpy()
    ds = ds.cpu().numpy()
    assert np.all(np.isfinite(s))
    err = np.abs(s - rs)
    assert np.all(err <= TOL_QP + 1e-5 * np.abs(rs)), f"max err {err.max():.3e}"
    assert np.all(np.abs(ds - rds) <= 1e-5 * (1 + np.abs(rds)))


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "tf32x3"])
def test_sigma_split_matches_fp64_gpu_path(prec):
    m = O.molecule("c1")
    ref = O.decomposition("c1", 1e-5)
    rov, rp = O.factors("c1", ref.L)
    E = W.energy_grid(m.eps[m.orbitals], 3, 0.02)
    a, _ = G.cds_sigma2_diag(dev(rov), dev(rp), dev(m.eps), m.nocc, dev(E), "fp64")
    b, _ = G.cds_sigma2_diag(dev(rov), dev(rp), dev(m.eps), m.nocc, dev(E), prec)
    assert np.abs(a.cpu().numpy() - b.cpu().numpy()).max() <= TOL_QP


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3", "tf32x3"])
@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_qp_split_within_tenth_of_mev(name, delta, prec):
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    rov, rp = O.factors(name, ref.L)
    w, P, it, st = G.cds_qp_solve(dev(rov), dev(rp), dev(m.orbitals), dev(m.eps), m.nocc,
                                  conv=1e-5, max_iter=50, precision=prec)
    res = O.solve(name, rov, rp, m.orbitals)
    w = w.cpu().numpy()
    st = st.cpu().numpy()
    for t, r in enumerate(res):
        assert st[t] == r[3]
        if r[3] == 0:
            assert abs(w[t] - r[0]) <= TOL_QP, (t, w[t], r[0])
            assert abs(P[t].item() - r[1]) <= 1e-4
