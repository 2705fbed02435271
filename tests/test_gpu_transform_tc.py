"""AO->MO transform on the tensor cores (Eq. transformation; tcgen05, split
precision) against the FP64 transform.

The FP64 transform is pinned against the oracle in test_gpu_parity.py (and
the oracle against the four-index transform).  The split-precision forms
accumulate in FP32, so their error is ~2^-21 (TF32X3) or ~2^-17 (BF16X3)
times the cancellation ratio sum|C||A||C| / |Lov|.  That ratio is small for
well-conditioned coefficients and ~1e6 for the ring and C60-shaped inputs,
whose C = S^-1/2 Q reaches |C| ~ 100-300 (cond ~1e4): there only the FP64
and float-pair forms are accurate, and the tensor-core form is an opt-in.
Here, on well-conditioned inputs:
* TF32X3 within 2e-6 and BF16X3 within 5e-5 of the largest |element|, on the
  tiny molecule (cond C = 7.7) and on random orthogonal C with N = 240 (eight
  k-blocks, two N tiles);
* ragged shapes: a rank that is not a multiple of the 32-vector batch, no
  requested orbitals, a single occupied orbital;
* the pipelined decomposition + transform with the tensor-core transform
  equals the separate calls' results to the same bound;
* the exact-slice form (OZAKI: six 7-bit BF16 slices per operand, exact
  FP32 sums of the leading slice pairs) within 2e-5 everywhere, also on the
  ring molecule, where the FP32-accumulated split form is off by more than
  1e-3.
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
TOL = {"tf32x3": 2e-6, "bf16x3": 5e-5, "ozaki": 2e-5}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel_err(x, ref):
    return ((x - ref).abs().max() / ref.abs().max()).item()


def random_case(N=240, nocc=40, M=70, seed=5):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((M, N * (N + 1) // 2))
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    orbs = np.array([0, nocc - 2, nocc - 1, nocc, nocc + 1, N - 1], dtype=np.int32)
    return dev(L), dev(Q), nocc, dev(orbs)


@pytest.fixture(scope="module", params=["c0", "random"])
def case(request):
    if request.param == "c0":
        m = O.molecule("c0")
        L, C, nocc, orbs = dev(O.decomposition("c0", m.delta).L), dev(m.C), m.nocc, dev(m.orbitals)
    else:
        L, C, nocc, orbs = random_case()
    Lov, Lp = G.cds_cd_to_mo(L, C, nocc, orbs, precision="fp64")
    return request.param, L, C, nocc, orbs, Lov, Lp


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "ozaki"])
def test_tc_transform_matches_fp64(case, prec):
    name, L, C, nocc, orbs, Lov, Lp = case
    Lov2, Lp2 = G.cds_cd_to_mo(L, C, nocc, orbs, precision=prec)
    e_ov, e_p = rel_err(Lov2, Lov), rel_err(Lp2, Lp)
    print(f"{name} {prec} M={L.shape[0]} Lov {e_ov:.2e} Lp {e_p:.2e}")
    assert e_ov <= TOL[prec] and e_p <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "ozaki"])
def test_tc_transform_ragged_shapes(case, prec):
    name, L, C, nocc, orbs, Lov, Lp = case
    # a rank that is not a multiple of the batch
    M = max(1, L.shape[0] - 5)
    a, b = G.cds_cd_to_mo(L[:M].contiguous(), C, nocc, orbs, precision=prec)
    assert rel_err(a, Lov[:, :, :M]) <= TOL[prec] and rel_err(b, Lp[:, :, :M]) <= TOL[prec]
    # no requested orbitals
    a, b = G.cds_cd_to_mo(L, C, nocc, orbs[:0], precision=prec)
    assert rel_err(a, Lov) <= TOL[prec] and b.numel() == 0
    # a single occupied orbital (one row block of T, ragged everywhere)
    a, b = G.cds_cd_to_mo(L, C, 1, orbs, precision=prec)
    ref_a, ref_b = G.cds_cd_to_mo(L, C, 1, orbs, precision="fp64")
    assert rel_err(a, ref_a) <= TOL[prec] and rel_err(b, ref_b) <= TOL[prec]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "ozaki"])
def test_fused_with_tc_transform(prec):
    m = O.molecule("c0")
    xyz, al, at = dev(m.basis.xyz), dev(m.basis.alpha), dev(m.basis.atom.astype(np.int32))
    C, orbs = dev(m.C), dev(m.orbitals)
    L, piv, D, de, Lov, Lp = G.cds_cd_decompose_to_mo(xyz, al, at, m.delta, C, m.nocc, orbs,
                                                      transform=prec)
    Lf, piv2, _, _ = G.cds_cd_decompose(xyz, al, at, m.delta, "full", precision="f32x2")
    assert torch.equal(piv, piv2)
    ref_ov, ref_p = G.cds_cd_to_mo(Lf, C, m.nocc, orbs, precision="fp64")
    assert rel_err(Lov, ref_ov) <= TOL[prec] and rel_err(Lp, ref_p) <= TOL[prec]


def test_ill_conditioned_coefficients():
    """Ring molecule (max|C| = 294, largest column 1-norm ~1.1e4, cancellation
    ratio ~1e6): the float-pair transform stays within 1e-7 of max|Lov| and
    the exact-slice tensor-core form within 2e-5, while the FP32-accumulated
    split forms refuse the call (CDS_ERR_UNSUPPORTED: u |C|_1^2 > 2^-8)
    instead of returning factors off by more than 1e-3."""
    m = O.molecule("c1")
    L = dev(O.decomposition("c1", m.delta).L[:64])
    C, orbs = dev(m.C), dev(m.orbitals)
    ref, ref_p = G.cds_cd_to_mo(L, C, m.nocc, orbs, precision="fp64")
    e_f2 = rel_err(G.cds_cd_to_mo(L, C, m.nocc, orbs, precision="f32x2")[0], ref)
    for prec in ("tf32x3", "bf16x3"):
        with pytest.raises(G.CdsError) as ei:
            G.cds_cd_to_mo(L, C, m.nocc, orbs, precision=prec)
        assert ei.value.status == 7
    oz_ov, oz_p = G.cds_cd_to_mo(L, C, m.nocc, orbs, precision="ozaki")
    e_oz, e_ozp = rel_err(oz_ov, ref), rel_err(oz_p, ref_p)
    print(f"ring: f32x2 {e_f2:.2e} ozaki {e_oz:.2e} / {e_ozp:.2e}")
    assert e_f2 <= 1e-7 and e_oz <= 2e-5 and e_ozp <= 2e-5


def test_exact_slice_rejects_bases_beyond_its_exactness_bound():
    """The leading slice pairs sum exactly in FP32 only for contraction
    lengths K <= 1040 (K 127^2 < 2^24): a larger basis is refused with
    CDS_ERR_UNSUPPORTED instead of losing the exactness silently; rank 0 is a
    no-op."""
    N = 1100
    L = torch.zeros((1, N * (N + 1) // 2), dtype=torch.float64, device=DEV)
    C = torch.eye(N, dtype=torch.float64, device=DEV)
    orbs = torch.tensor([0, 1], dtype=torch.int32, device=DEV)
    with pytest.raises(G.CdsError):
        G.cds_cd_to_mo(L, C, 10, orbs, precision="ozaki")
    m = O.molecule("c0")
    a, b = G.cds_cd_to_mo(torch.zeros((0, G.npair(m.nbf)), dtype=torch.float64, device=DEV),
                          dev(m.C), m.nocc, dev(m.orbitals), precision="ozaki")
    assert a.numel() == 0 and b.numel() == 0
