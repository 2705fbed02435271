"""GPU path against the CPU oracle, element by element, through the C ABI.

Tolerances (FP64 path): integrals 1e-13 relative; Cholesky vectors and
residuals 1e-11 absolute (values <= 2, about k*1e-16 of accumulated rounding
after k steps); MO factors 1e-11 relative to their largest entry;
self-energy, its derivative and the Newton roots 1e-10 Ha.  Pivot sequences
must be identical (ties inside the 1e-12 band resolve to the same lowest
index on both sides).  Sizes span several tiles and ragged tails: o = 6, 40,
v = 18, 200 against 32-row blocks.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import eri
from tests import oracle_pipeline as O

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0912_1459_gb300 as G  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def basis_dev(m):
    return dev(m.basis.xyz), dev(m.basis.alpha), dev(m.basis.atom.astype(np.int32))


def gpu_cd(m, delta, scheme="full", max_rank=None, precision="fp64"):
    xyz, a, at = basis_dev(m)
    L, piv, D, de = G.cds_cd_decompose(xyz, a, at, delta, scheme, max_rank=max_rank,
                                       precision=precision)
    torch.cuda.synchronize()
    return L.cpu().numpy(), piv.cpu().numpy().astype(np.int64), D.cpu().numpy(), de


@pytest.mark.parametrize("name", ["c0", "c1"])
def test_eri_diag_and_columns(name):
    m = O.molecule(name)
    pd = O.pairs(name)
    xyz, a, _ = basis_dev(m)
    D = G.cds_eri_diag(xyz, a).cpu().numpy()
    np.testing.assert_allclose(D, eri.eri_diagonal(pd), rtol=1e-13, atol=1e-150)
    rng = np.random.default_rng(0)
    piv = rng.choice(pd.npair, 5, replace=False).astype(np.int32)
    cols = G.cds_eri_columns(xyz, a, dev(piv)).cpu().numpy()
    for c, P in enumerate(piv):
        ref = eri.eri_column(pd, int(P))
        np.testing.assert_allclose(cols[c], ref, rtol=1e-13, atol=1e-150)


@pytest.mark.parametrize("name,delta,scheme", [
    ("c0", 1e-6, "full"), ("c0", 1e-3, "full"), ("c0", 0.0, "full"), ("c0", 1e-6, "atomic"),
    ("c1", 1e-4, "full"), ("c1", 1e-5, "full"), ("c1", 1e-6, "full"), ("c1", 1e-4, "atomic"),
    ("c1", 1e-6, "atomic"),
])
def test_cd_parity(name, delta, scheme):
    m = O.molecule(name)
    ref = O.decomposition(name, delta, scheme)
    L, piv, D, de = gpu_cd(m, delta, scheme)
    assert de == pytest.approx(ref.delta_eff, rel=1e-14)
    assert len(piv) == ref.M
    assert np.array_equal(piv, ref.piv)
    # rows pivoted on residuals far above roundoff agree element by element;
    # rows pivoted on residuals near delta_eff ~ 1e-13 (delta = 0) are rounding
    # noise amplified by 1/sqrt(D_P) and are checked through the product L^T L
    dp = ref.L[np.arange(ref.M), ref.piv] ** 2
    sharp = dp >= 1e-9 * ref.scale
    np.testing.assert_allclose(L[sharp], ref.L[sharp], rtol=0, atol=1e-11)
    sub = np.random.default_rng(1).choice(L.shape[1], min(L.shape[1], 600), replace=False)
    np.testing.assert_allclose(L[:, sub].T @ L[:, sub], ref.L[:, sub].T @ ref.L[:, sub],
                               rtol=0, atol=1e-11)
    np.testing.assert_allclose(D, ref.D, rtol=0, atol=1e-11)


@pytest.mark.parametrize("name,delta,scheme", [
    ("c0", 1e-6, "full"), ("c1", 1e-4, "full"), ("c1", 1e-6, "full"), ("c1", 1e-5, "atomic"),
])
def test_cd_f32x2_parity(name, delta, scheme):
    """Float-pair projections (~2^-44 per step instead of 2^-53): the same
    pivots as the oracle, vectors and residuals within 1e-9, L^T L within
    1e-9 on sampled pairs."""
    m = O.molecule(name)
    ref = O.decomposition(name, delta, scheme)
    L, piv, D, de = gpu_cd(m, delta, scheme, precision="f32x2")
    assert de == pytest.approx(ref.delta_eff, rel=1e-14)
    assert np.array_equal(piv, ref.piv)
    np.testing.assert_allclose(L, ref.L, rtol=0, atol=1e-9)
    sub = np.random.default_rng(2).choice(L.shape[1], min(L.shape[1], 600), replace=False)
    np.testing.assert_allclose(L[:, sub].T @ L[:, sub], ref.L[:, sub].T @ ref.L[:, sub],
                               rtol=0, atol=1e-9)
    np.testing.assert_allclose(D, ref.D, rtol=0, atol=1e-9)


@pytest.mark.parametrize("name,delta,scheme", [
    ("c0", 1e-6, "full"), ("c0", 1e-6, "atomic"), ("c1", 1e-4, "full"), ("c1", 1e-5, "full"),
    ("c1", 1e-6, "full"), ("c1", 1e-5, "atomic"),
])
def test_cd_tensor_core_parity(name, delta, scheme):
    """Exact-slice tensor-core passes (CDS_PREC_OZAKI: the stored vectors as
    56-bit fixed point below each pair's scale sigma_I > sqrt(D0_I), 32
    candidates per pass): the oracle's pivots; vectors within
    tol = max(1e-9, 1e-11 / sqrt(delta)) -- a projection carries ~2^-56
    sigma_I sigma_P k of truncation plus the shared accumulator's rounding
    (~1e-14 sigma_I sigma_P), and L^k divides it by sqrt(D_P) >= sqrt(delta);
    the bound keeps the 42-bit analysis' margin; L^T L and the residuals
    within the same."""
    m = O.molecule(name)
    ref = O.decomposition(name, delta, scheme)
    L, piv, D, de = gpu_cd(m, delta, scheme, precision="ozaki")
    tol = max(1e-9, 1e-11 / np.sqrt(delta))
    assert de == pytest.approx(ref.delta_eff, rel=1e-14)
    assert np.array_equal(piv, ref.piv)
    np.testing.assert_allclose(L, ref.L, rtol=0, atol=tol)
    sub = np.random.default_rng(2).choice(L.shape[1], min(L.shape[1], 600), replace=False)
    np.testing.assert_allclose(L[:, sub].T @ L[:, sub], ref.L[:, sub].T @ ref.L[:, sub],
                               rtol=0, atol=tol)
    np.testing.assert_allclose(D, ref.D, rtol=0, atol=tol)


def test_cd_tensor_core_screening():
    """Screening of the tensor-core form: the pairs kept are exactly those
    with D0_I >= 1e-40 max D0 (oracle diagonal); the others return L = 0 and
    their initial diagonal, and every kept pair matches the oracle."""
    m = O.molecule("c1")
    ref = O.decomposition("c1", 1e-5, "full")
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    D0 = eri.eri_diagonal(pd)
    live = D0 >= 1e-40 * D0.max()
    assert 0 < live.sum() < pd.npair          # the ring has negligible pairs
    xyz, a, at = dev(m.basis.xyz), dev(m.basis.alpha), dev(m.basis.atom.astype(np.int32))
    lib = G.load()
    ws = torch.empty(lib.cds_cd_workspace_bytes_prec(m.nbf, 1024, 6), dtype=torch.uint8,
                     device=DEV)
    L, piv, D, de = G.cds_cd_decompose(xyz, a, at, 1e-5, "full", max_rank=1024, workspace=ws,
                                       precision="ozaki")
    torch.cuda.synchronize()
    assert G.cdsigma.cds_cd_live_pairs(m.nbf, ws, "ozaki") == int(live.sum())
    L, D = L.cpu().numpy(), D.cpu().numpy()
    assert np.array_equal(piv.cpu().numpy().astype(np.int64), ref.piv)
    assert not L[:, ~live].any()
    np.testing.assert_allclose(D[~live], D0[~live], rtol=1e-12, atol=1e-30 * D0.max())
    np.testing.assert_allclose(L[:, live], ref.L[:, live], rtol=0, atol=1e-9)
    assert np.abs(ref.L[:, ~live]).max() <= 1e-19     # what screening leaves out


def test_cd_tensor_core_chunk_graph():
    """On a stream of its own (not a default stream) and with max_rank >= 512
    the tensor-core decomposition replays each 32-step chunk as one CUDA
    graph, the step number read from the device: the oracle's pivots and
    the same vectors as the step-by-step launches (bit for bit), with the
    graph switched on and off through CDS_TUNE_CD_GRAPH."""
    m = O.molecule("c1")
    ref = O.decomposition("c1", 1e-5, "full")
    xyz, a, at = dev(m.basis.xyz), dev(m.basis.alpha), dev(m.basis.atom.astype(np.int32))
    s = torch.cuda.Stream()
    out = {}
    try:
        for knob in (512, 0):
            G.cdsigma.cds_tune_set(G.cdsigma.TUNE_CD_GRAPH, knob)
            with torch.cuda.stream(s):
                L, piv, D, de = G.cds_cd_decompose(xyz, a, at, 1e-5, "full", max_rank=1024,
                                                   precision="ozaki")
            s.synchronize()
            out[knob] = (L.cpu().numpy(), piv.cpu().numpy().astype(np.int64), D.cpu().numpy())
    finally:
        G.cdsigma.cds_tune_set(G.cdsigma.TUNE_CD_GRAPH, 512)
    assert np.array_equal(out[512][1], ref.piv)
    assert np.array_equal(out[512][0], out[0][0]) and np.array_equal(out[512][2], out[0][2])
    np.testing.assert_allclose(out[512][0], ref.L, rtol=0, atol=1e-9)


def test_cd_tensor_core_refuses_bases_beyond_its_candidate_search():
    """The tensor-core form keeps the update blocks' maxima in shared memory:
    more than 2048 blocks of 512 pairs left after screening (here every pair
    of 1460 diffuse functions in a 20-bohr cube is kept) is refused before
    the first step with CDS_ERR_UNSUPPORTED."""
    n = 1460
    rng = np.random.default_rng(0)
    xyz = dev(rng.uniform(0, 20, (n, 3)))
    a = dev(np.full(n, 0.05))
    at = dev(np.arange(n, dtype=np.int32))
    with pytest.raises(G.CdsError) as ei:
        G.cds_cd_decompose(xyz, a, at, 1e-4, "full", max_rank=1, precision="ozaki")
    assert ei.value.status == 7


def test_cd_precision_rejected():
    m = O.molecule("c0")
    with pytest.raises(G.CdsError) as ei:
        gpu_cd(m, 1e-6, precision="bf16x3")
    assert ei.value.status == 7


def test_cd_empty_when_delta_exceeds_every_diagonal():
    m = O.molecule("c0")
    L, piv, D, de = gpu_cd(m, 100.0)
    assert L.shape[0] == 0 and piv.shape[0] == 0
    np.testing.assert_allclose(D, eri.eri_diagonal(O.pairs("c0")), rtol=1e-13)


def test_cd_rank_cap_reports_and_keeps_prefix():
    m = O.molecule("c0")
    xyz, a, at = basis_dev(m)
    with pytest.raises(G.CdsError) as ei:
        G.cds_cd_decompose(xyz, a, at, 1e-6, "full", max_rank=10)
    assert ei.value.status == 4
    L = torch.empty((10, G.npair(m.nbf)), dtype=torch.float64, device=DEV)
    with pytest.raises(G.CdsError):
        G.cds_cd_decompose(xyz, a, at, 1e-6, "full", max_rank=10, L_out=L)
    ref = O.decomposition("c0", 1e-6, "full")
    np.testing.assert_allclose(L.cpu().numpy(), ref.L[:10], rtol=0, atol=1e-12)


@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_transform_parity(name, delta):
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    orbs = np.concatenate([m.orbitals, [0, m.nbf - 1]]).astype(np.int32)
    Lov, Lp = G.cds_cd_to_mo(dev(ref.L), dev(m.C), m.nocc, dev(orbs))
    rov, rp = O.factors(name, ref.L, orbs)
    scale = max(np.abs(rov).max(), np.abs(rp).max())
    np.testing.assert_allclose(Lov.cpu().numpy(), rov, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(Lp.cpu().numpy(), rp, rtol=0, atol=1e-11 * scale)


@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_transform_float_pairs(name, delta):
    """F32X2 transform against the oracle within 1e-10 (|C|^T |A| |C|)_pq: the
    float-pair arithmetic carries ~2^-44 per operation over N terms."""
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    orbs = m.orbitals.astype(np.int32)
    Lov, Lp = G.cds_cd_to_mo(dev(ref.L), dev(m.C), m.nocc, dev(orbs), precision="f32x2")
    rov, rp = O.factors(name, ref.L, orbs)
    from oracle import ao2mo
    absC = np.abs(m.C)
    Lov, Lp = Lov.cpu().numpy(), Lp.cpu().numpy()
    for K in range(0, ref.M, max(1, ref.M // 7)):
        bound = absC.T @ np.abs(ao2mo.unpack(ref.L[K], m.nbf)) @ absC
        assert np.all(np.abs(Lov[:, :, K] - rov[:, :, K]) <= 1e-10 * bound[:m.nocc, m.nocc:])
        assert np.all(np.abs(Lp[:, :, K] - rp[:, :, K]) <= 1e-10 * bound[orbs, :])


@pytest.mark.parametrize("name,delta,nE", [("c0", 1e-6, 16), ("c1", 1e-5, 4)])
def test_sigma_fp64_parity(name, delta, nE):
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    rov, rp = O.factors(name, ref.L)
    E = W.energy_grid(m.eps[m.orbitals], nE)
    s, ds = G.cds_sigma2_diag(dev(rov), dev(rp), dev(m.eps), m.nocc, dev(E), "fp64")
    rs, rds = O.sigma(name, rov, rp, E)
    np.testing.assert_allclose(s.cpu().numpy(), rs, rtol=0, atol=1e-10)
    np.testing.assert_allclose(ds.cpu().numpy(), rds, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("name,delta", [("c0", 1e-6), ("c1", 1e-5)])
def test_qp_fp64_parity(name, delta):
    m = O.molecule(name)
    ref = O.decomposition(name, delta)
    rov, rp = O.factors(name, ref.L)
    w, P, it, st = G.cds_qp_solve(dev(rov), dev(rp), dev(m.orbitals), dev(m.eps), m.nocc,
                                  conv=1e-5, max_iter=50, precision="fp64")
    res = O.solve(name, rov, rp, m.orbitals)
    np.testing.assert_allclose(w.cpu().numpy(), [r[0] for r in res], rtol=0, atol=1e-10)
    np.testing.assert_allclose(P.cpu().numpy(), [r[1] for r in res], rtol=1e-9, atol=0)
    assert it.cpu().tolist() == [r[2] for r in res]
    assert st.cpu().tolist() == [r[3] for r in res]


def test_end_to_end_tiny_pipeline():
    """CD -> transform -> Sigma -> Newton entirely on the GPU vs entirely in the oracle."""
    m = O.molecule("c0")
    xyz, a, at = basis_dev(m)
    L, piv, D, de = G.cds_cd_decompose(xyz, a, at, m.delta, "full")
    Lov, Lp = G.cds_cd_to_mo(L, dev(m.C), m.nocc, dev(m.orbitals))
    E = W.energy_grid(m.eps[m.orbitals], m.nE)
    s, ds = G.cds_sigma2_diag(Lov, Lp, dev(m.eps), m.nocc, dev(E), "fp64")
    w, P, it, st = G.cds_qp_solve(Lov, Lp, dev(m.orbitals), dev(m.eps), m.nocc)
    ref = O.decomposition("c0", m.delta)
    rov, rp = O.factors("c0", ref.L)
    rs, _ = O.sigma("c0", rov, rp, E)
    res = O.solve("c0", rov, rp, m.orbitals)
    np.testing.assert_allclose(s.cpu().numpy(), rs, atol=1e-10, rtol=0)
    np.testing.assert_allclose(w.cpu().numpy(), [r[0] for r in res], atol=1e-10, rtol=0)


def test_sigma_edge_cases():
    m = O.molecule("c0")
    ref = O.decomposition("c0", 1e-6)
    # every orbital, one energy each: occupied and virtual q, ragged single block
    orbs = np.arange(m.nbf, dtype=np.int32)
    rov, rp = O.factors("c0", ref.L, orbs)
    E = m.eps[:, None] + 0.013
    s, ds = G.cds_sigma2_diag(dev(rov), dev(rp), dev(m.eps), m.nocc, dev(E), "fp64")
    rs, rds = O.sigma("c0", rov, rp, E)
    np.testing.assert_allclose(s.cpu().numpy(), rs, atol=1e-10, rtol=0)
    # no orbitals: a no-op
    s0, _ = G.cds_sigma2_diag(dev(rov), dev(rp[:0]), dev(m.eps), m.nocc, dev(E[:0]), "fp64")
    assert s0.shape == (0, 1)
    # a single Cholesky vector
    rov1, rp1 = O.factors("c0", ref.L[:1], orbs[:3])
    s1, _ = G.cds_sigma2_diag(dev(rov1), dev(rp1), dev(m.eps), m.nocc, dev(E[:3]), "fp64")
    rs1, _ = O.sigma("c0", rov1, rp1, E[:3])
    np.testing.assert_allclose(s1.cpu().numpy(), rs1, atol=1e-12, rtol=0)


def test_tiny_case_against_stored_oracle_values():
    """The whole FP64 path on the tiny case against tests/golden/c0_oracle.json."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "c0_oracle.json")) as f:
        g = json.load(f)
    m = O.molecule("c0")
    xyz, a, at = basis_dev(m)
    L, piv, D, de = G.cds_cd_decompose(xyz, a, at, g["delta"], "full")
    assert piv.cpu().tolist() == g["cd"]["piv"]
    orbs = dev(np.asarray(g["orbitals"], dtype=np.int32))
    Lov, Lp = G.cds_cd_to_mo(L, dev(m.C), m.nocc, orbs)
    eps = dev(m.eps)
    E = dev(m.eps[g["orbitals"]][:, None])
    s, ds = G.cds_sigma2_diag(Lov, Lp, eps, m.nocc, E, "fp64")
    np.testing.assert_allclose(s.cpu().numpy()[:, 0], g["sigma_at_eps"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(ds.cpu().numpy()[:, 0], g["dsigma_at_eps"], rtol=1e-9)
    w, P, it, st = G.cds_qp_solve(Lov, Lp, orbs, eps, m.nocc, precision="fp64")
    for t, r in enumerate(g["qp"]):
        assert int(it[t]) == r["iters"] and int(st[t]) == r["status"]
        assert float(w[t]) == pytest.approx(r["omega"], abs=1e-9)
        assert float(P[t]) == pytest.approx(r["pole"], rel=1e-8)


@pytest.mark.parametrize("precision", ["fp64", "f32x2", "ozaki"])
def test_cd_stats_counters(precision):
    """cds_cd_stats: FP64 streams at every step; the speculative forms stream
    at the first step of each batch of at most B steps (4 for float pairs, 64
    on the tensor cores, whose passes project 32 candidates), and a continued
    step adds between one and B-1 vectors."""
    m = O.molecule("c1")
    xyz, a, at = basis_dev(m)
    prec = G.cdsigma.PRECISIONS[precision]
    ws = torch.empty(G.load().cds_cd_workspace_bytes_prec(m.nbf, 1024, prec), dtype=torch.uint8,
                     device=DEV)
    L, piv, D, de = G.cds_cd_decompose(xyz, a, at, 1e-5, "full", max_rank=1024, workspace=ws,
                                       precision=precision)
    M = L.shape[0]
    st = G.cdsigma.cds_cd_stats(m.nbf, ws, precision)
    ncand = G.cdsigma.cd_candidates(precision)
    if precision == "fp64":
        assert ncand == 1
        assert st == {"passes": M, "streamed": M * (M - 1) // 2, "extra": 0}
    else:
        assert ncand == {"f32x2": 4, "ozaki": 32}[precision]
        B = {"f32x2": 4, "ozaki": 64}[precision]
        assert (M + B - 1) // B <= st["passes"] <= M
        assert 0 < st["streamed"] < M * (M - 1) // 2
        cont = M - st["passes"]
        assert cont <= st["extra"] <= (B - 1) * cont


@pytest.mark.parametrize("cdp", ["f32x2", "ozaki"])
@pytest.mark.parametrize("name,delta,orbs", [("c1", 1e-5, None), ("c0", 1e-6, []), ("c1", 1e-4, [39, 40])])
def test_fused_decompose_to_mo_matches_separate_calls(name, delta, orbs, cdp):
    """cds_cd_decompose_to_mo (float-pair CD with the transform overlapped) gives
    the pivots and vectors of cds_cd_decompose(F32X2) and the factors of
    cds_cd_to_mo(F32X2) on them.  The pipelined transform reads the float-pair
    rows directly, the separate one their FP64 conversion, whose rounding the
    transform's cancellation (|C| ~ 1e3) magnifies: 1e-8 of the largest entry."""
    m = O.molecule(name)
    xyz, a, at = basis_dev(m)
    orb = dev(np.asarray(m.orbitals if orbs is None else orbs, dtype=np.int32))
    L1, piv1, D1, de1 = G.cds_cd_decompose(xyz, a, at, delta, "full", precision=cdp)
    Lov1, Lp1 = G.cds_cd_to_mo(L1, dev(m.C), m.nocc, orb, precision="f32x2")
    L2, piv2, D2, de2, Lov2, Lp2 = G.cds_cd_decompose_to_mo(xyz, a, at, delta, dev(m.C), m.nocc,
                                                           orb, cd_precision=cdp)
    assert torch.equal(piv1, piv2) and torch.equal(L1, L2) and torch.equal(D1, D2)
    assert Lov2.shape == Lov1.shape and Lp2.shape == Lp1.shape
    scale = Lov1.abs().max().item()
    assert (Lov1 - Lov2).abs().max().item() <= 1e-8 * scale
    if Lp1.numel():
        assert (Lp1 - Lp2).abs().max().item() <= 1e-8 * Lp1.abs().max().item()


def test_fused_rank_cap_rows_are_fp64():
    """A pipelined tensor-core call stopped by its rank cap (CDS_ERR_RANK_CAP)
    at 40 vectors: the last, partial batch of rows is transformed and
    converted to FP64 at the stop, so L equals the standalone decomposition's
    (which converts all rows at its end) and the factors match the separate
    transform's."""
    m = O.molecule("c1")
    xyz, a, at = basis_dev(m)
    orb = dev(np.asarray(m.orbitals, dtype=np.int32))
    cap, npr = 40, G.npair(m.nbf)
    L1 = torch.empty((cap, npr), dtype=torch.float64, device=DEV)
    with pytest.raises(G.CdsError) as ei:
        G.cds_cd_decompose(xyz, a, at, 1e-6, "full", max_rank=cap, L_out=L1, precision="ozaki")
    assert ei.value.status == 4
    L2 = torch.empty((cap, npr), dtype=torch.float64, device=DEV)
    nv = m.nbf - m.nocc
    Lov2 = torch.empty(m.nocc * nv * cap, dtype=torch.float64, device=DEV)
    Lp2 = torch.empty(len(m.orbitals) * m.nbf * cap, dtype=torch.float64, device=DEV)
    with pytest.raises(G.CdsError) as ei:
        G.cds_cd_decompose_to_mo(xyz, a, at, 1e-6, dev(m.C), m.nocc, orb, max_rank=cap,
                                 L_out=L2, Lov_out=Lov2, Lp_out=Lp2, transform="ozaki",
                                 cd_precision="ozaki")
    assert ei.value.status == 4
    assert torch.equal(L1, L2)
    Lov1, Lp1 = G.cds_cd_to_mo(L1, dev(m.C), m.nocc, orb, precision="ozaki")
    Lov2 = Lov2[:m.nocc * nv * cap].view(m.nocc, nv, cap)
    scale = Lov1.abs().max().item()
    assert (Lov1 - Lov2).abs().max().item() <= 1e-8 * scale
