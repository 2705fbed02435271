"""Small, self-contained cases for profiling one kernel at a time.

Each case builds only the inputs of one library call at C60 shape (N = 840,
o = 180, v = 660) and runs it twice, so an ``ncu -k <kernel> -c <n>`` capture
holds a few GB of device memory at most and replays in seconds:

  python -m paper_0912_1459_gb300.profcases transform   # k_dfgemm (float pairs)
  python -m paper_0912_1459_gb300.profcases transform_oz  # k_oz_gemm, k_oz_slice (exact slices)
  python -m paper_0912_1459_gb300.profcases sigma1      # k_sigma_tc, nE = 1
  python -m paper_0912_1459_gb300.profcases sigma64     # k_sigma_tc, nE = 64
  python -m paper_0912_1459_gb300.profcases grid        # k_sigma_tc (nE = 1, keeps the
                                                        # numerators), k_sigma_cached_grid (63)
  python -m paper_0912_1459_gb300.profcases cd          # k_cd_update, FP64 (C60, 1024 steps max)
  python -m paper_0912_1459_gb300.profcases cdf         # k_cd_update, float pairs
  python -m paper_0912_1459_gb300.profcases cdoz        # k_cd_gemm_tc, k_cd_project_tc,
                                                        # k_cd_update (tensor-core passes; 512
                                                        # steps, 4.4 GB on the device)
  python -m paper_0912_1459_gb300.profcases bcd         # batched tensor-core decomposition of
                                                        # the 64 clusters (launch lists only:
                                                        # ~70 GB on the device)
  python -m paper_0912_1459_gb300.profcases bcd8        # the same for 8 clusters of 240..300
                                                        # functions, rank capacity 640 (8 GB)

Factors are seeded random numbers of the right shape and magnitude (the
kernels' cost does not depend on their values).
"""
from __future__ import annotations

import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

from . import cdsigma as G  # noqa: E402


def main(mode: str) -> None:
    dev = torch.device("cuda:0")

    def d(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    m = W.config2()
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    if mode in ("transform", "transform64", "transform_oz"):
        L = torch.randn((128, G.npair(m.nbf)), dtype=torch.float64, device=dev, generator=g) * 1e-2
        prec = {"transform64": "fp64", "transform_oz": "ozaki"}.get(mode, "f32x2")
        for rep in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            G.cds_cd_to_mo(L, d(m.C), m.nocc, d(m.orbitals), precision=prec)
            b.record()
            torch.cuda.synchronize()
            print(f"transform of {L.shape[0]} vectors: {a.elapsed_time(b):.2f} ms")
    elif mode == "grid":
        Lov = torch.randn((m.nocc, m.nbf - m.nocc, 896), dtype=torch.float64, device=dev,
                          generator=g) * 1e-2
        Lp = torch.randn((2, m.nbf, 896), dtype=torch.float64, device=dev, generator=g) * 1e-2
        E = d(W.energy_grid(m.eps[m.orbitals[9:11]], 64))
        for _ in range(2):
            G.cds_sigma2_diag_cache(Lov, Lp, d(m.eps), m.nocc, E, "bf16x3")
    elif mode in ("sigma1", "sigma64"):
        nE = 64 if mode == "sigma64" else 1
        Lov = torch.randn((m.nocc, m.nbf - m.nocc, 896), dtype=torch.float64, device=dev,
                          generator=g) * 1e-2
        Lp = torch.randn((2, m.nbf, 896), dtype=torch.float64, device=dev, generator=g) * 1e-2
        E = d(W.energy_grid(m.eps[m.orbitals[9:11]], nE))
        for _ in range(2):
            G.cds_sigma2_diag(Lov, Lp, d(m.eps), m.nocc, E, "bf16x3")
    elif mode in ("cd", "cdf", "cdoz"):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rank = 512 if mode == "cdoz" else 1024
        try:
            L, _, _, _ = G.cds_cd_decompose(d(m.basis.xyz), d(m.basis.alpha),
                                            d(m.basis.atom.astype(np.int32)), 1e-4, "full",
                                            max_rank=rank,
                                            precision={"cdf": "f32x2", "cdoz": "ozaki"}.get(
                                                mode, "fp64"))
            M = L.shape[0]
        except G.CdsError as e:   # the first `rank` steps are all a profile needs
            if e.status != 4:
                raise
            M = rank
        b.record()
        torch.cuda.synchronize()
        print(f"decomposition: {M} steps, {a.elapsed_time(b):.1f} ms")
    elif mode in ("bcd", "bcd8"):
        mols = W.config3()
        cap = None
        if mode == "bcd8":
            mols = [c for c in mols if 240 <= c.nbf <= 300][:8]
            cap = 640
        spec = [(c.nbf, c.nocc, len(c.orbitals), c.nE, cap or G.default_max_rank(c.nbf))
                for c in mols]
        bt = G.Batch(spec, dev, "bf16x3", cd_precision="ozaki")

        def cat(xs):
            return d(np.concatenate(xs))
        xyz = cat([c.basis.xyz.ravel() for c in mols])
        al = cat([c.basis.alpha for c in mols])
        at = cat([c.basis.atom.astype(np.int32) for c in mols])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        M = bt.cd_decompose(xyz, al, at, mols[0].delta, precision="ozaki")
        b.record()
        torch.cuda.synchronize()
        print(f"batched decomposition of {len(mols)} clusters (ranks {min(M)}..{max(M)}): "
              f"{a.elapsed_time(b):.1f} ms")
    else:
        raise SystemExit(f"unknown case {mode!r}")
    torch.cuda.synchronize()
    print("ok", mode)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "sigma1")
