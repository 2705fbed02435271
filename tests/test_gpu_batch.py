"""Batched form (many molecules per call) against the single-molecule calls
and the oracle.

Eight clusters of the batched workload (centre counts U{4..40}, 10
s-Gaussians each, o = N/5, delta = 1e-5, U{4..16} orbitals on U{8..64}
energies).  The batch reproduces the single-molecule results: the same
pivots and Cholesky vectors, the same transform, the self-energy and Newton
results of the same kernels within 1e-12 (only the order items are
scheduled in differs; Newton from the cached numerators, and with the
recomputing passes), and one molecule against the FP64 oracle within the
mixed-precision bar.  The captured CUDA graph replays to the same results,
twice in a row.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import ao2mo, cd, eri, qp, sigma2

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0912_1459_gb300 as G  # noqa: E402
from paper_0912_1459_gb300 import cdsigma as C  # noqa: E402

DEV = torch.device("cuda:0")
TOL_QP = 0.1e-3 / 27.211396


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def batch():
    mols = W.config3()[:8]
    spec = [(m.nbf, m.nocc, len(m.orbitals), m.nE, C.default_max_rank(m.nbf)) for m in mols]
    b = C.Batch(spec, DEV, "bf16x3")
    cat = lambda xs: dev(np.concatenate(xs))  # noqa: E731
    xyz = cat([m.basis.xyz.ravel() for m in mols])
    al = cat([m.basis.alpha for m in mols])
    at = cat([m.basis.atom.astype(np.int32) for m in mols])
    Cc = cat([m.C.ravel() for m in mols])
    eps = cat([m.eps for m in mols])
    orb = cat([m.orbitals.astype(np.int32) for m in mols])
    E = cat([W.energy_grid(m.eps[m.orbitals], m.nE).ravel() for m in mols])
    M = b.cd_decompose(xyz, al, at, mols[0].delta)
    b.cd_to_mo(Cc, orb, precision="f32x2")
    b.sigma2(eps, E)
    b.qp_solve(orb, eps)
    torch.cuda.synchronize()
    return mols, b, M, dict(xyz=xyz, al=al, at=at, C=Cc, eps=eps, orb=orb, E=E)


def single(m, cached=True):
    L, piv, D, de = G.cds_cd_decompose(dev(m.basis.xyz), dev(m.basis.alpha),
                                       dev(m.basis.atom.astype(np.int32)), m.delta, "full")
    Lov, Lp = G.cds_cd_to_mo(L, dev(m.C), m.nocc, dev(m.orbitals), precision="f32x2")
    E = dev(W.energy_grid(m.eps[m.orbitals], m.nE))
    s, ds, cache = G.cds_sigma2_diag_cache(Lov, Lp, dev(m.eps), m.nocc, E, "bf16x3")
    if cached:
        w, P, it, st = G.cds_qp_solve_cached(cache, dev(m.orbitals), dev(m.eps), m.nbf, m.nocc)
    else:
        w, P, it, st = G.cds_qp_solve(Lov, Lp, dev(m.orbitals), dev(m.eps), m.nocc,
                                      precision="bf16x3")
    return L, piv, Lov, Lp, s, w, P, it, st


def test_batch_matches_single_molecule_calls(batch):
    mols, b, M, inp = batch
    for c, m in enumerate(mols):
        L, piv, Lov, Lp, s, w, P, it, st = single(m)
        npr = G.npair(m.nbf)
        assert M[c] == L.shape[0]
        assert torch.equal(b.view("piv", c, (M[c],)), piv)
        torch.testing.assert_close(b.view("L", c, (M[c], npr)), L, rtol=0, atol=1e-11)
        nv, np_ = m.nbf - m.nocc, len(m.orbitals)
        torch.testing.assert_close(b.view("ov", c, (m.nocc, nv, M[c])), Lov, rtol=0, atol=1e-12)
        torch.testing.assert_close(b.view("p", c, (np_, m.nbf, M[c])), Lp, rtol=0, atol=1e-12)
        torch.testing.assert_close(b.view("sigma", c, (np_, m.nE)), s, rtol=1e-12, atol=1e-12)
        torch.testing.assert_close(b.view("omega", c, (np_,)), w, rtol=0, atol=1e-12)
        assert torch.equal(b.view("iters", c, (np_,)), it)
        assert torch.equal(b.view("status", c, (np_,)), st)


def test_batch_recomputing_newton_matches_single_calls(batch):
    """CDS_TUNE_NEWTON_CACHE = 0: the batched Newton passes recompute the
    integrals, like cds_qp_solve."""
    mols, b, M, inp = batch
    G.cdsigma.cds_tune_set(G.cdsigma.TUNE_NEWTON_CACHE, 0)
    try:
        b.sigma2(inp["eps"], inp["E"])
        b.qp_solve(inp["orb"], inp["eps"])
        torch.cuda.synchronize()
        for c, m in enumerate(mols):
            *_, w, P, it, st = single(m, cached=False)
            np_ = len(m.orbitals)
            torch.testing.assert_close(b.view("omega", c, (np_,)), w, rtol=0, atol=1e-12)
            assert torch.equal(b.view("status", c, (np_,)), st)
    finally:
        G.cdsigma.cds_tune_set(G.cdsigma.TUNE_NEWTON_CACHE, 1)
        b.sigma2(inp["eps"], inp["E"])
        b.qp_solve(inp["orb"], inp["eps"])
        torch.cuda.synchronize()


def test_batch_molecule_against_oracle(batch):
    mols, b, M, inp = batch
    c = int(np.argmin([m.nbf for m in mols]))
    m = mols[c]
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    ref = cd.decompose(pd, m.delta)
    assert M[c] == ref.M
    rov, rp = ao2mo.mo_factors(ref.L, m.C, m.nocc, m.orbitals)
    E = W.energy_grid(m.eps[m.orbitals], m.nE)
    np_ = len(m.orbitals)
    got = b.view("sigma", c, (np_, m.nE)).cpu().numpy()
    w = b.view("omega", c, (np_,)).cpu().numpy()
    for t, q in enumerate(m.orbitals):
        rs, _ = sigma2.sigma2_from_factors(rp[t], rov, m.eps, m.nocc, E[t])
        assert np.all(np.abs(got[t] - rs) <= TOL_QP + 1e-5 * np.abs(rs))

        def f(x, t=t):
            a, d = sigma2.sigma2_from_factors(rp[t], rov, m.eps, m.nocc, [x])
            return a[0], d[0]
        wr, Pr, itr, str_ = qp.newton_qp(f, m.eps[q])
        if str_ == 0 and Pr >= 0.5:
            assert abs(w[t] - wr) <= TOL_QP


def test_graph_replays_reproduce_the_direct_calls(batch):
    mols, b, M, inp = batch
    sig0, w0 = b.sigma.clone(), b.omega.clone()
    it0 = b.iters.clone()
    g = b.graph(inp["orb"], inp["eps"], inp["E"])
    for _ in range(2):
        b.sigma.fill_(float("nan"))
        b.omega.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        torch.testing.assert_close(b.sigma, sig0, rtol=0, atol=0)
        torch.testing.assert_close(b.omega, w0, rtol=0, atol=0)
        assert torch.equal(b.iters, it0)
    st = b.stamps.cpu().numpy()
    assert np.all(st[1:] >= st[0]) and np.all(st[1:] > 0)
    del g


def test_autotuner_candidates_agree_and_cache(batch, tmp_path, monkeypatch):
    from paper_0912_1459_gb300 import autotune
    mols, b, M, inp = batch
    monkeypatch.setenv("CDS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    results = {}
    for cand in autotune.CANDIDATES:
        autotune.apply(cand)
        g = b.graph(inp["orb"], inp["eps"], inp["E"])
        g.launch()
        torch.cuda.synchronize()
        results[cand] = (b.sigma.clone(), b.omega.clone(), b.pole.clone(), b.status.clone())
        del g
    for cand, (s_, w_, p_, st_) in results.items():
        # items are reduced per orbital in a fixed order, so the chunk, the
        # order and the grid kernel's energies per pass change only which CTA
        # or which pass computes a value, not the arithmetic
        ref = results[(16, 0, cand[2], 4)]
        torch.testing.assert_close(s_, ref[0], rtol=1e-13, atol=1e-13)
        torch.testing.assert_close(w_, ref[1], rtol=1e-13, atol=1e-13)
    # Newton from the kept numerators against recomputed integrals: the same
    # per-element arithmetic, FP32 sums in another order -- the grid within
    # 1e-5 relative, quasiparticle roots (P >= 0.5, converged) within 1e-7 Ha
    a, r = results[(16, 0, 1, 4)], results[(16, 0, 0, 4)]
    torch.testing.assert_close(a[0], r[0], rtol=1e-5, atol=1e-8)
    qp = (a[3] == 0) & (r[3] == 0) & (r[2] >= 0.5)
    assert int(qp.sum()) >= 10
    assert (a[1] - r[1])[qp].abs().max().item() <= 1e-7
    first = autotune.tune(b, inp["orb"], inp["eps"], inp["E"])
    assert first["cached"] is False and tuple(first["choice"]) in autotune.CANDIDATES
    again = autotune.tune(b, inp["orb"], inp["eps"], inp["E"])
    assert again["cached"] is True and tuple(again["choice"]) == tuple(first["choice"])
    autotune.apply((16, 0, 1, 4))


def test_batch_exact_slice_transform(batch):
    """The batched transform with the exact-slice tensor-core form (ozaki):
    every molecule's Lov / Lp within 5e-5 of its largest entry of the
    float-pair transform (42-bit slices against the cancellation of
    C = S^-1/2 Q); the float-pair results are restored afterwards."""
    mols, b, M, inp = batch
    ref = [(b.view("ov", c, (m.nocc, m.nbf - m.nocc, M[c])).clone(),
            b.view("p", c, (len(m.orbitals), m.nbf, M[c])).clone()) for c, m in enumerate(mols)]
    try:
        b.cd_to_mo(inp["C"], inp["orb"], precision="ozaki")
        torch.cuda.synchronize()
        for c, m in enumerate(mols):
            ov = b.view("ov", c, (m.nocc, m.nbf - m.nocc, M[c]))
            p = b.view("p", c, (len(m.orbitals), m.nbf, M[c]))
            assert (ov - ref[c][0]).abs().max().item() <= 5e-5 * ref[c][0].abs().max().item()
            assert (p - ref[c][1]).abs().max().item() <= 5e-5 * ref[c][1].abs().max().item()
    finally:
        b.cd_to_mo(inp["C"], inp["orb"], precision="f32x2")
        torch.cuda.synchronize()


def test_batch_float_pair_decomposition(batch):
    """The batched decomposition in float pairs (float-pair projections and
    vectors; FP64 column, residuals and pivot decisions) against the FP64
    batch: every molecule's pivots identical, vectors within 1e-8 (the
    single-molecule float-pair bar)."""
    mols, b, M, inp = batch
    spec = [(m.nbf, m.nocc, len(m.orbitals), m.nE, C.default_max_rank(m.nbf)) for m in mols]
    bf = C.Batch(spec, DEV, "bf16x3")
    Mf = bf.cd_decompose(inp["xyz"], inp["al"], inp["at"], mols[0].delta, precision="f32x2")
    torch.cuda.synchronize()
    assert Mf == M
    for c, m in enumerate(mols):
        npr = G.npair(m.nbf)
        assert torch.equal(bf.view("piv", c, (M[c],)), b.view("piv", c, (M[c],)))
        torch.testing.assert_close(bf.view("L", c, (M[c], npr)), b.view("L", c, (M[c], npr)),
                                   rtol=0, atol=1e-8)


def test_batch_tensor_core_decomposition(batch):
    """The batched decomposition with the tensor-core passes (every
    molecule's screening, then three launches per step for the whole batch)
    against the FP64 batch: every molecule's pivots identical, vectors within
    1e-9 (the single-molecule tensor-core bar); and against the
    single-molecule tensor-core call: the same arithmetic per molecule, so
    pivots, vectors and residuals bit for bit."""
    mols, b, M, inp = batch
    spec = [(m.nbf, m.nocc, len(m.orbitals), m.nE, C.default_max_rank(m.nbf)) for m in mols]
    bt = C.Batch(spec, DEV, "bf16x3", cd_precision="ozaki")
    Mt = bt.cd_decompose(inp["xyz"], inp["al"], inp["at"], mols[0].delta, precision="ozaki")
    torch.cuda.synchronize()
    assert Mt == M
    for c, m in enumerate(mols):
        npr = G.npair(m.nbf)
        assert torch.equal(bt.view("piv", c, (M[c],)), b.view("piv", c, (M[c],)))
        torch.testing.assert_close(bt.view("L", c, (M[c], npr)), b.view("L", c, (M[c], npr)),
                                   rtol=0, atol=1e-9)
    for c in (0, 3, 7):
        m = mols[c]
        npr = G.npair(m.nbf)
        L1, p1, D1, _ = G.cds_cd_decompose(dev(m.basis.xyz), dev(m.basis.alpha),
                                           dev(m.basis.atom.astype(np.int32)), m.delta, "full",
                                           precision="ozaki")
        assert L1.shape[0] == M[c]
        assert torch.equal(bt.view("piv", c, (M[c],)), p1)
        assert torch.equal(bt.view("L", c, (M[c], npr)), L1)
        assert torch.equal(bt.view("D", c, (npr,)), D1)


def test_batch_tensor_core_atomic(batch):
    """The atomic pivot restriction (Sec. II.A) in the batched tensor-core
    form: pivots identical to the FP64 batch, every pivot a one-centre pair,
    vectors within 1e-9."""
    mols, _, _, inp = batch
    spec = [(m.nbf, m.nocc, len(m.orbitals), m.nE, C.default_max_rank(m.nbf)) for m in mols]
    b64 = C.Batch(spec, DEV, "bf16x3")
    M64 = b64.cd_decompose(inp["xyz"], inp["al"], inp["at"], mols[0].delta, "atomic")
    bt = C.Batch(spec, DEV, "bf16x3", cd_precision="ozaki")
    Mt = bt.cd_decompose(inp["xyz"], inp["al"], inp["at"], mols[0].delta, "atomic",
                         precision="ozaki")
    torch.cuda.synchronize()
    assert Mt == M64
    for c, m in enumerate(mols):
        npr = G.npair(m.nbf)
        pv = bt.view("piv", c, (Mt[c],))
        assert torch.equal(pv, b64.view("piv", c, (Mt[c],)))
        mu, nu = eri.pair_list(m.nbf)
        p = pv.cpu().numpy()
        assert np.all(m.basis.atom[mu[p]] == m.basis.atom[nu[p]])
        torch.testing.assert_close(bt.view("L", c, (Mt[c], npr)), b64.view("L", c, (Mt[c], npr)),
                                   rtol=0, atol=1e-9)


def test_batch_tensor_core_many_molecules():
    """More molecules than one batched launch takes (1024): the batch runs in
    groups.  1030 small clusters (1..3 centres, seeded), pivots identical to
    the FP64 batch and vectors within 1e-9."""
    rng = np.random.default_rng(11)
    nmol = 1030
    xyz, al, at, spec, nbfs = [], [], [], [], []
    for c in range(nmol):
        nat = int(rng.integers(1, 4))
        cen = rng.uniform(0.0, 3.0, (nat, 3))
        ex = W.geometric_exponents(0.2, 6.0, 4)
        for a in range(nat):
            for e in ex:
                xyz.append(cen[a])
                al.append(e)
                at.append(a)
        nbf = 4 * nat
        nbfs.append(nbf)
        spec.append((nbf, 1, 1, 1, C.default_max_rank(nbf)))
    xyz = dev(np.array(xyz).ravel())
    al = dev(np.array(al))
    at = dev(np.array(at, dtype=np.int32))
    b64 = C.Batch(spec, DEV, "bf16x3")
    M64 = b64.cd_decompose(xyz, al, at, 1e-6)
    bt = C.Batch(spec, DEV, "bf16x3", cd_precision="ozaki")
    Mt = bt.cd_decompose(xyz, al, at, 1e-6, precision="ozaki")
    torch.cuda.synchronize()
    assert Mt == M64
    for c in list(range(0, nmol, 97)) + [1023, 1024, 1029]:
        npr = G.npair(nbfs[c])
        assert torch.equal(bt.view("piv", c, (Mt[c],)), b64.view("piv", c, (Mt[c],)))
        torch.testing.assert_close(bt.view("L", c, (Mt[c], npr)), b64.view("L", c, (Mt[c], npr)),
                                   rtol=0, atol=1e-9)


def test_batch_tensor_core_degenerate_molecules():
    """Edge cases in one batched tensor-core call, against the FP64 batch:
    a single function (one pair), a molecule whose diagonal is below delta
    from the start (rank 0), two coincident functions (a rank-deficient
    supermatrix), and an ordinary cluster."""
    rng = np.random.default_rng(5)
    parts = []   # (xyz [n,3], alpha [n], atom [n])
    parts.append((np.zeros((1, 3)), np.array([0.9]), np.zeros(1, np.int32)))
    parts.append((np.array([[0.0, 0, 0], [0.5, 0, 0]]), np.array([1e-7, 2e-7]),
                  np.zeros(2, np.int32)))
    parts.append((np.array([[0.0, 0, 0], [0.0, 0, 0], [1.2, 0, 0]]), np.array([0.7, 0.7, 1.3]),
                  np.array([0, 0, 1], np.int32)))
    cen = rng.uniform(0, 4, (5, 3))
    ex = W.geometric_exponents(0.2, 6.0, 4)
    parts.append((np.repeat(cen, 4, axis=0), np.tile(ex, 5), np.repeat(np.arange(5), 4).astype(np.int32)))
    spec = [(len(p[1]), 0, 1, 1, C.default_max_rank(len(p[1]))) for p in parts]
    xyz = dev(np.concatenate([p[0].ravel() for p in parts]))
    al = dev(np.concatenate([p[1] for p in parts]))
    at = dev(np.concatenate([p[2] for p in parts]))
    delta = 1e-3
    b64 = C.Batch(spec, DEV, "bf16x3")
    M64 = b64.cd_decompose(xyz, al, at, delta)
    bt = C.Batch(spec, DEV, "bf16x3", cd_precision="ozaki")
    Mt = bt.cd_decompose(xyz, al, at, delta, precision="ozaki")
    torch.cuda.synchronize()
    assert Mt == M64
    assert Mt[0] == 1 and Mt[1] == 0 and Mt[2] < G.npair(3)
    for c, p in enumerate(parts):
        npr = G.npair(len(p[1]))
        assert torch.equal(bt.view("piv", c, (Mt[c],)), b64.view("piv", c, (Mt[c],)))
        torch.testing.assert_close(bt.view("L", c, (Mt[c], npr)), b64.view("L", c, (Mt[c], npr)),
                                   rtol=0, atol=1e-9)
        torch.testing.assert_close(bt.view("D", c, (npr,)), b64.view("D", c, (npr,)),
                                   rtol=0, atol=1e-9)
