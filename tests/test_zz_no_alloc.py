"""The allocation-free decomposition entry point (cds_cd_decompose_static).

It serves callers that cannot allocate device memory where they call: it
takes inputs and outputs only and works in a fixed scratch array inside the
library.  Checked through the C ABI against the workspace entry point
(cds_cd_decompose) on the same inputs, for two calls in a row (the shared
array keeps the previous call's contents, which must not leak into the
next result), with the tolerances of the Cholesky parity tests: identical
pivots, vectors and residuals within 1e-11.  The second call must leave the
device's free memory and torch's pool unchanged.  Collected last so a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_0912_1459_gb300 as G  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_static_entry_point_matches_workspace_entry_point_twice():
    m = W.config1()                      # N = 240, within the static capacity
    assert m.nbf <= G.load().cds_cd_static_max_nbf()
    xyz, al, at = dev(m.basis.xyz), dev(m.basis.alpha), dev(m.basis.atom.astype(np.int32))
    cases = [(1e-5, "full"), (1e-4, "atomic")]
    for delta, scheme in cases:
        L, piv, D, de = G.cds_cd_decompose(xyz, al, at, delta, scheme, max_rank=1024)
        Lr, pr, Dr = L.cpu().numpy(), piv.cpu().numpy(), D.cpu().numpy()
        npr = G.npair(m.nbf)
        for call in range(2):
            Ls = torch.full((1024, npr), float("nan"), dtype=torch.float64, device=DEV)
            ps = torch.full((1024,), -1, dtype=torch.int32, device=DEV)
            Ds = torch.full((npr,), float("nan"), dtype=torch.float64, device=DEV)
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info(DEV)[0]
            held0 = torch.cuda.memory_reserved(DEV)
            M, de_s = G.cdsigma.cds_cd_decompose_static(xyz, al, at, delta, scheme, Ls, ps, Ds)
            torch.cuda.synchronize()
            if call == 1:   # after the first call (module and kernels loaded): no device memory taken
                assert torch.cuda.mem_get_info(DEV)[0] >= free0
                assert torch.cuda.memory_reserved(DEV) == held0
            assert M == Lr.shape[0]
            assert de_s == de
            assert np.array_equal(ps[:M].cpu().numpy(), pr)
            np.testing.assert_allclose(Ls[:M].cpu().numpy(), Lr, rtol=0, atol=1e-11)
            np.testing.assert_allclose(Ds.cpu().numpy(), Dr, rtol=0, atol=1e-11)


def test_static_entry_point_rejects_too_large_basis():
    m = W.config2()                      # N = 840 needs more than the fixed scratch
    assert m.nbf > G.load().cds_cd_static_max_nbf()
    npr = G.npair(m.nbf)
    L = torch.empty((1, npr), dtype=torch.float64, device=DEV)
    piv = torch.empty((1,), dtype=torch.int32, device=DEV)
    D = torch.empty((npr,), dtype=torch.float64, device=DEV)
    with pytest.raises(G.CdsError) as ei:
        G.cdsigma.cds_cd_decompose_static(dev(m.basis.xyz), dev(m.basis.alpha),
                                          dev(m.basis.atom.astype(np.int32)), 1e-4, "full",
                                          L, piv, D)
    assert ei.value.status == 9
