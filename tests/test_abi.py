"""The C-ABI library loads without a GPU and exports every declared entry point."""
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_0912_1459_gb300", "libcdsigma.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_0912_1459_gb300 import build as b
        b.build()
    from paper_0912_1459_gb300 import cdsigma
    return cdsigma


def test_every_declared_symbol_is_exported(lib):
    names = lib.declared_symbols()
    assert "cds_cd_decompose" in names and "cds_sigma2_diag" in names and "cds_qp_solve" in names
    so = lib.load()
    missing = [n for n in names if not hasattr(so, n)]
    assert missing == []


def test_host_only_calls(lib):
    so = lib.load()
    assert so.cds_version() >= 100
    assert so.cds_errstr(4).decode().startswith("Cholesky rank cap")
    assert so.cds_cd_workspace_bytes(24) > 300 * 5 * 8
    assert so.cds_cd_workspace_bytes(-1) == 0
    assert so.cds_sigma2_workspace_bytes(24, 6, 100, 2, 16, 0) > 0
    assert so.cds_sigma2_workspace_bytes(24, 6, 100, 2, 0, 0) == 0
    # the GEMM timing switch and totals are host state only
    lib.cds_cd_gemm_timing(True)
    assert lib.cds_cd_gemm_time() == (0.0, 0)
    lib.cds_cd_gemm_timing(False)


def test_argument_errors_before_any_launch(lib):
    so = lib.load()
    # invalid sizes are rejected on the host, without touching a device
    assert so.cds_cd_decompose(0, None, None, None, 1e-6, 0, 10, 0, None, None, None, None, None,
                               None, 0, None) == 1
    assert so.cds_sigma2_diag(24, 6, 10, None, None, 1, None, None, 0, 0, None, None, None, 0,
                              None) == 1
    assert so.cds_sigma2_diag(24, 6, 10, None, None, 1, None, None, 4, 9, None, None, None, 0,
                              None) == 7
    assert so.cds_qp_solve(24, 6, 10, None, None, None, 1, None, 1e-5, 0, 0, None, None, None,
                           None, None, 0, None) == 1


def test_batch_workspace_sizes(lib):
    """Host-side sizing of the batched workspace.  The tensor-core
    decomposition (CDS_PREC_OZAKI) adds its own region after the worker slots.
    The region holds every molecule's slice store: 8 BF16 slices per pair and
    column of max_rank rounded up to 32, and more besides.  The transform's
    workspace grows with the number of vectors up to its batch size."""
    so = lib.load()
    spec = [(40, 8, 4, 8, 240), (120, 24, 6, 16, 512), (7, 1, 1, 1, 28)]
    mols = (lib.CdsMol * len(spec))(*[lib.CdsMol(*m) for m in spec])
    other = so.cds_batch_workspace_bytes(len(spec), mols, lib.PRECISIONS["bf16x3"])
    oz = so.cds_batch_workspace_bytes(len(spec), mols, lib.PRECISIONS["ozaki"])
    assert other > 0
    stores = sum(16 * lib.npair(n) * ((r + 31) // 32 * 32) for n, _, _, _, r in spec)
    assert oz - other >= stores
    assert so.cds_batch_workspace_bytes(0, mols, lib.PRECISIONS["ozaki"]) == 0
    # the transform: more vectors need more room, up to the batch size
    w = [so.cds_cd_to_mo_workspace_bytes(100, 100, 20, m, 4) for m in (1, 32, 320, 700, 2000)]
    assert w[0] <= w[1] <= w[2] <= w[3] == w[4]
