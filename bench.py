#!/usr/bin/env python3
"""Benchmark: C60-shaped Sigma(2) quasiparticle solves per second on GB300.

One step = the whole hot path on the C60-shaped workload (60-centre
truncated-icosahedron cage, 14 s-Gaussians per centre, N = 840, o = 180,
v = 660), inputs resident in HBM:
  1. threshold-delta pivoted Cholesky decomposition of the ERI supermatrix
     (full scheme, delta = 1e-4, on-the-fly columns),
  2. AO->MO transform of the Cholesky vectors,
  3. Sigma_qq(E) and dSigma/dE for 20 orbitals around the gap on 64 energies,
  4. Newton quasiparticle solve of the same 20 orbitals (Delta = 1e-5).
value = quasiparticle solves per second of the whole step (20 per step).

Also reported: per-stage times, a roofline entry per stage, the same metric
end to end from pinned host buffers (e2e), the FP64 GPU path for the
self-energy stages on a subset of orbitals, the accuracy of the mixed path
against it, and a CPU-oracle baseline on a bounded sample.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs an independent replica (the path has no
exchange step; weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "C60-shaped Sigma(2) QP solves/s (whole step: CD + AO->MO + Sigma grid + Newton)"
UNIT = "solves/s"
WORKLOAD = "c60-shaped N=840 o=180 v=660 (truncated icosahedron, 14 s-Gaussians/centre)"
HARTREE_EV = 27.211396     # Sec. III conversion factor
L2_BYTES = 129 * 2 ** 20


def parse():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp16x3", "tf32x3", "fp64"])
    p.add_argument("--delta", type=float, default=1e-4)
    p.add_argument("--scheme", default="full", choices=["full", "atomic"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-arm", action="store_true",
                   help="skip the measured all-FP64 GPU step and the per-orbital accuracy tables")
    p.add_argument("--no-adjoint", action="store_true",
                   help="skip timing the adjoint of 8 gap orbitals")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-mp2", action="store_true")
    p.add_argument("--transform", default="ozaki", choices=["ozaki", "f32x2"],
                   help="transform of the pipelined step: exact-slice tcgen05 GEMMs or "
                        "float-pair GEMMs on the FP32 units")
    p.add_argument("--cd-precision", default="ozaki", choices=["f32x2", "ozaki"],
                   help="decomposition of the pipelined step: speculative float-pair passes (4 "
                        "candidates) or exact-slice tensor-core passes (32 candidates)")
    p.add_argument("--no-trtc", action="store_true",
                   help="skip timing the other transform forms on the step's vectors")
    p.add_argument("--no-acd", action="store_true",
                   help="skip the atomic-Cholesky-basis / V-approximation section")
    p.add_argument("--no-fuse", action="store_true",
                   help="run the decomposition and the transform as two calls (stage times "
                        "of each) instead of the pipelined cds_cd_decompose_to_mo")
    p.add_argument("--newton", default="cached", choices=["cached", "recompute"],
                   help="Newton from the numerators the Sigma-grid stage keeps, or recomputing "
                        "the integrals every iteration (split precisions)")
    return p.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (replicas only)
# ----------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float, device) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def done(self):
        if self.pg:
            self.pg.destroy_process_group()


def host_cores() -> int:
    """Host threads available to this process (numpy's BLAS uses all of them)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def aggregate_value(world: int, solves_per_step: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput of N replicas: every rank solves the same number of
    orbitals per step; the slowest rank's time (max over ranks) bounds the job."""
    return world * solves_per_step * steps / (max_ms / 1e3)


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def workload(delta: float):
    m = W.config2(delta=delta)
    E = W.energy_grid(m.eps[m.orbitals], m.nE)
    return m, E


def flops_model(m, M: int) -> dict:
    """Algorithmic work per call (the units of the roofline entries)."""
    N, o = m.nbf, m.nocc
    v, n_orb = m.nbf - o, len(m.orbitals)
    npair = N * (N + 1) // 2
    return {
        # left-looking CD: sum_k 2 k npair flops (projections) -> npair M^2
        "cd": float(npair) * M * M,
        # bytes: step k reads k stored vectors (8 B each per pair) and writes
        # one; with the residual diagonal (read + write), the pair data (5
        # doubles) and the candidate mask and the selection's re-read of the
        # diagonal, 8 k + 73 bytes per pair per step
        "cd_bytes": float(npair) * (4.0 * M * (M - 1) + 73.0 * M),
        # C_occ^T A C_vir and C_P^T A C per vector
        "transform": 2.0 * M * (o * N * (N + v) + n_orb * N * (N + N)),
        # one Sigma pass per orbital: X for both sums, 2 M (o v^2 + v o^2)
        "sigma_pass": 2.0 * M * (o * v * v + v * o * o),
    }


CD_GEMM_TRAFFIC_PER_BYTE = 1.837708936e9 / 1.838065024e9


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    meas = {}
    if os.path.exists(path):
        with open(path) as f:
            meas = json.load(f)
    return {
        "bf16_tflops": meas.get("bf16_tflops", 1900.0),
        "bf16_tflops_sustained": meas.get("bf16_tflops_sustained", 1700.0),
        "hbm_gbs": meas.get("hbm_gbs", 6800.0),
        "source": "measured" if meas else "fallback",
        # FP64 and FP32 issue rates: nominal GB300 figures (an FMA-throughput
        # probe on this pool measured 1.25 and 78 TFLOP/s)
        "fp64_tflops": 1.25,
        "fp32_tflops": 78.0,
        # FP32 instruction issue: 152 SMs x 128 lanes x 2.07 GHz (nominal clock)
        "fp32_issue_tinstr": 152 * 128 * 2.07e9 / 1e12,
    }


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args, dist: Dist):
    import torch
    import paper_0912_1459_gb300 as G

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (no CPU fallback)")
    device = torch.device("cuda", dist.local)
    torch.cuda.set_device(device)
    dist.init("nccl")
    prec = args.precision
    # the split-precision pipeline decomposes and transforms in float pairs,
    # the FP64 one in FP64
    tr_prec = "fp64" if prec == "fp64" else "f32x2"
    m, Egrid = workload(args.delta)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
    xyz, al, at = d(m.basis.xyz), d(m.basis.alpha), d(m.basis.atom.astype(np.int32))
    C, eps, orbs, E = d(m.C), d(m.eps), d(m.orbitals), d(Egrid)
    n_orb = len(m.orbitals)
    lib = G.load()

    # device buffers reused by every step
    max_rank = 2048 if args.delta >= 1e-5 else 4096
    npr = G.npair(m.nbf)
    Lbuf = torch.empty((max_rank, npr), dtype=torch.float64, device=device)
    cd_ws = torch.empty(lib.cds_cd_workspace_bytes_prec(m.nbf, max_rank, G.cdsigma.PRECISIONS[
        args.cd_precision if prec != "fp64" else "fp64"]), dtype=torch.uint8, device=device)
    cached = args.newton == "cached" and prec != "fp64"
    cache = (torch.empty(lib.cds_sigma2_cache_bytes(m.nbf, m.nocc, n_orb, G.cdsigma.PRECISIONS[prec]), dtype=torch.uint8,
                         device=device) if cached else None)

    fused = not args.no_fuse and tr_prec != "fp64"
    if fused:
        nv = m.nbf - m.nocc
        lov_buf = torch.empty(m.nocc * nv * max_rank, dtype=torch.float64, device=device)
        lp_buf = torch.empty(n_orb * m.nbf * max_rank, dtype=torch.float64, device=device)
        fz_ws = torch.empty(lib.cds_cd_decompose_to_mo_workspace_bytes(
                                m.nbf, m.nbf, m.nocc, max_rank, n_orb,
                                G.cdsigma.PRECISIONS[args.cd_precision]),
                            dtype=torch.uint8, device=device)

    def step(xyz, al, at, C, eps, orbs, E, ws=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record()
        if fused:
            # decomposition and transform pipelined in one call: one stage
            L, piv, D, de, Lov, Lp = G.cds_cd_decompose_to_mo(
                xyz, al, at, args.delta, C, m.nocc, orbs, args.scheme, L_out=Lbuf,
                Lov_out=lov_buf, Lp_out=lp_buf, workspace=fz_ws, transform=args.transform,
                cd_precision=args.cd_precision)
            ev[1].record()
            ev[2].record()
        else:
            L, piv, D, de = G.cds_cd_decompose(xyz, al, at, args.delta, args.scheme, L_out=Lbuf,
                                               workspace=cd_ws, precision=tr_prec)
            ev[1].record()
            Lov, Lp = G.cds_cd_to_mo(L, C, m.nocc, orbs, workspace=ws and ws.get("tr"),
                                     precision=tr_prec)
            ev[2].record()
        if cached:
            sig, dsig, _ = G.cds_sigma2_diag_cache(Lov, Lp, eps, m.nocc, E, prec, cache=cache,
                                                   workspace=ws and ws.get("sg"))
            ev[3].record()
            w, P, it, st = G.cds_qp_solve_cached(cache, orbs, eps, m.nbf, m.nocc, conv=1e-5,
                                                 max_iter=50, workspace=ws and ws.get("qpc"))
        else:
            sig, dsig = G.cds_sigma2_diag(Lov, Lp, eps, m.nocc, E, prec,
                                          workspace=ws and ws.get("sg"))
            ev[3].record()
            w, P, it, st = G.cds_qp_solve(Lov, Lp, orbs, eps, m.nocc, conv=1e-5, max_iter=50,
                                          precision=prec, workspace=ws and ws.get("qp"))
        ev[4].record()
        return (L, Lov, Lp, sig, dsig, w, P, it, st), ev

    # warm-up (also sizes the per-stage workspaces once)
    out, _ = step(xyz, al, at, C, eps, orbs, E)
    M = out[0].shape[0]
    ws = {
        "tr": torch.empty(lib.cds_cd_to_mo_workspace_bytes(m.nbf, m.nbf, m.nocc, M, n_orb),
                          dtype=torch.uint8, device=device),
        "sg": torch.empty(lib.cds_sigma2_workspace_bytes(m.nbf, m.nocc, M, n_orb, m.nE,
                                                          G.cdsigma.PRECISIONS[prec]),
                          dtype=torch.uint8, device=device),
        "qp": torch.empty(lib.cds_qp_workspace_bytes(m.nbf, m.nocc, M, n_orb,
                                                      G.cdsigma.PRECISIONS[prec]),
                          dtype=torch.uint8, device=device),
        "qpc": torch.empty(max(lib.cds_qp_cached_workspace_bytes(m.nbf, m.nocc, n_orb), 1),
                           dtype=torch.uint8, device=device),
    }
    for _ in range(max(args.warmup - 1, 0)):
        out, _ = step(xyz, al, at, C, eps, orbs, E, ws)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs (all > L2: L is GBs) ----
    clocks = Clocks(device.index if device.index is not None else 0)
    # the tensor-core decomposition's projection GEMM, the step's dominant
    # kernel, is timed by the library with CUDA events around each of its
    # launches, on the stream it launches on, in extra steps after the timed
    # ones (the 1,792 event records of a step would slow the timed steps' host
    # loop by ~4 %)
    gemm_timed = fused and args.cd_precision == "ozaki"
    dist.barrier()
    torch.cuda.synchronize()
    launches0 = G.cds_launch_count()
    clocks.start()
    torch.cuda.nvtx.range_push("timed")      # lets a profiler select exactly the timed steps
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    stage_ms = {"cd": [], "transform": [], "sigma_grid": [], "qp": []}
    evs = []
    for _ in range(args.steps):
        out, ev = step(xyz, al, at, C, eps, orbs, E, ws)
        evs.append(ev)
    t1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    dist.barrier()
    clk = clocks.stop()
    launches = G.cds_launch_count() - launches0
    if gemm_timed:
        G.cdsigma.cds_cd_gemm_timing(True)
        for _ in range(args.steps):
            step(xyz, al, at, C, eps, orbs, E, ws)
        torch.cuda.synchronize()
        gemm_ms, gemm_launches = G.cdsigma.cds_cd_gemm_time()
        # the same kernel with the decomposition alone (no transform beside it)
        G.cdsigma.cds_cd_gemm_timing(True)
        G.cds_cd_decompose(xyz, al, at, args.delta, args.scheme, L_out=Lbuf, workspace=cd_ws,
                           precision="ozaki")
        torch.cuda.synchronize()
        gemm_alone_ms, gemm_alone_launches = G.cdsigma.cds_cd_gemm_time()
        G.cdsigma.cds_cd_gemm_timing(False)
    elapsed_ms = t0.elapsed_time(t1)
    for ev in evs:
        for k, (a, b) in zip(stage_ms, [(0, 1), (1, 2), (2, 3), (3, 4)]):
            stage_ms[k].append(ev[a].elapsed_time(ev[b]))
    elapsed_ms = dist.max(elapsed_ms, device)
    L, Lov, Lp, sig, dsig, w, P, it, st = out
    M = L.shape[0]
    value = aggregate_value(dist.world, n_orb, args.steps, elapsed_ms)

    # ---- end to end: pinned host inputs -> results on the host ----
    host_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
               for a in (m.basis.xyz, m.basis.alpha, m.basis.atom.astype(np.int32), m.C, m.eps,
                         m.orbitals, Egrid)]
    h2d = sum(t.numel() * t.element_size() for t in host_in)
    host_out = [torch.empty(tuple(x.shape), dtype=x.dtype).pin_memory() for x in (sig, dsig, w, P, it, st)]
    d2h = sum(t.numel() * t.element_size() for t in host_out)
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        dev_in = [t.to(device, non_blocking=True) for t in host_in]
        res, _ = step(*dev_in, ws)
        for h, x in zip(host_out, (res[3], res[4], res[5], res[6], res[7], res[8])):
            h.copy_(x, non_blocking=True)
        torch.cuda.current_stream(device).synchronize()
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = dist.max(e0.elapsed_time(e1), device)
    e2e_value = aggregate_value(dist.world, n_orb, args.steps, e2e_ms)

    # ---- rooflines (per call, CUDA events on the launching stream) ----
    fm = flops_model(m, M)
    cd_stats = G.cdsigma.cds_cd_stats(m.nbf, fz_ws if fused else cd_ws,
                                      args.cd_precision if tr_prec != "fp64" else "fp64")
    cd_bytes = float(npr) * (8.0 * cd_stats["streamed"] + 8.0 * cd_stats["extra"] +
                             32.0 * cd_stats["passes"] + 89.0 * M)
    pk = peaks()
    iters = it.cpu().numpy()
    med = {k: max(statistics.median(v), 1e-6) for k, v in stage_ms.items()}
    sig_passes_grid = n_orb
    sig_passes_qp = int(iters.sum())
    split = 1 if prec == "fp64" else 3
    roof = {}
    if tr_prec == "fp64":
        roof["cd"] = {"bound": "alu", "unit": "TFLOP/s", "peak": pk["fp64_tflops"],
                      "achieved": fm["cd"] / (med["cd"] / 1e3) / 1e12,
                      "note": "FP64 projections npair*M^2 flops; peak = nominal FP64 rate"}
    else:
        roof["cd"] = {"bound": "hbm", "unit": "GB/s", "peak": pk["hbm_gbs"],
                      "achieved": cd_bytes / (med["cd"] / 1e3) / 1e9,
                      "note": (f"speculative float-pair projections: {cd_stats['passes']} "
                               f"streaming passes over {M} steps read {cd_stats['streamed']} "
                               f"stored vectors in total; bytes = npair*(8*streamed + "
                               f"8*extra + 32*passes + 89*M); stage time of k_cd_project_spec "
                               f"+ k_cd_update"),
                      "cd_stats": cd_stats,
                      "plain_left_looking_bytes": fm["cd_bytes"]}
    if tr_prec == "fp64":
        roof["transform"] = {"bound": "alu", "unit": "TFLOP/s", "peak": pk["fp64_tflops"],
                             "achieved": fm["transform"] / (med["transform"] / 1e3) / 1e12,
                             "note": "FP64 GEMMs; peak = nominal FP64 rate"}
    else:
        # float-pair multiply-add = 11 FP32 instructions (see csrc/ao2mo.cu)
        roof["transform"] = {"bound": "alu", "unit": "TFLOP/s", "peak": pk["fp32_tflops"] / 11.0,
                             "achieved": fm["transform"] / (med["transform"] / 1e3) / 1e12,
                             "note": "float-pair GEMMs; peak = FP32 FMA rate / 11 instructions "
                                     "per pair multiply-add, in FP64-equivalent flops"}
    sig_flops_grid = split * fm["sigma_pass"] * sig_passes_grid
    roof["sigma_grid"] = {"bound": "alu" if prec != "fp64" else "alu", "unit": "TFLOP/s",
                          "peak": pk["bf16_tflops"] if prec != "fp64" else pk["fp64_tflops"],
                          "achieved": sig_flops_grid / (med["sigma_grid"] / 1e3) / 1e12,
                          "note": "64 energies: the fused denominator epilogue (fp32/MUFU) bounds it"}
    sig_flops_qp = split * fm["sigma_pass"] * sig_passes_qp
    if cached:
        per_orb = lib.cds_sigma2_cache_bytes(m.nbf, m.nocc, n_orb, G.cdsigma.PRECISIONS[prec]) / n_orb
        roof["qp"] = {"bound": "hbm", "unit": "GB/s", "peak": pk["hbm_gbs"],
                      "achieved": sig_passes_qp * per_orb / (med["qp"] / 1e3) / 1e9,
                      "note": f"{sig_passes_qp} Sigma passes (nE=1) from cached numerators, "
                              f"{per_orb / 1e6:.0f} MB streamed per orbital pass"}
    else:
        roof["qp"] = {"bound": "tensor" if prec != "fp64" else "alu", "unit": "TFLOP/s",
                      "peak": pk["bf16_tflops"] if prec != "fp64" else pk["fp64_tflops"],
                      "achieved": sig_flops_qp / (med["qp"] / 1e3) / 1e12,
                      "note": f"{sig_passes_qp} Sigma passes (nE=1); {split} split products per MAC"}
    if fused and gemm_timed:
        # the pairs the tensor-core form kept after screening
        nlive = G.cdsigma.cds_cd_live_pairs(m.nbf, fz_ws, "ozaki")
        # one stage for both: the decomposition's HBM bytes (slice store read by
        # the passes, the float-pair extras, the per-step column / vector /
        # residual traffic) over the live pairs; the transform runs on the
        # tensor pipe beside it
        stage_bytes = float(nlive) * (16.0 * cd_stats["streamed"] + 8.0 * cd_stats["extra"] +
                                      89.0 * M)
        med["cd_transform"] = med.pop("cd")
        med.pop("transform")
        roof.pop("cd")
        roof.pop("transform")
        roof["cd_transform"] = {
            "bound": "hbm", "unit": "GB/s", "peak": pk["hbm_gbs"],
            "achieved": stage_bytes / (med["cd_transform"] / 1e3) / 1e9,
            "note": (f"pipelined decomposition (tensor-core passes) + exact-slice transform: "
                     f"bytes = nlive*(16*streamed + 8*extra + 89*M) ({nlive} live of {npr} "
                     f"pairs, {cd_stats['passes']} passes, {cd_stats['streamed']} vectors "
                     f"streamed, {cd_stats['extra']} extra); the transform's slice-pair GEMMs run "
                     f"on the tensor pipe beside it"),
            "cd_stats": cd_stats}
        # the dominant kernel: k_cd_gemm_tc, per launch.  Algorithmic bytes of
        # a decomposition: the slice store (8 BF16 slices = 16 bytes per pair
        # and stored vector) read once per pass, the candidates' slices
        # (16 bytes x 32 per vector), the projections written (32 float pairs
        # = 256 bytes per pair) and the pair scales read (4 bytes per pair) at
        # every pass with k0 > 0
        gemm_bytes = (16.0 * nlive * cd_stats["streamed"] + 512.0 * cd_stats["streamed"] +
                      260.0 * nlive * max(cd_stats["passes"] - 1, 0))
        per_launch = gemm_bytes * args.steps / max(gemm_launches, 1)
        avg_ms = gemm_ms / max(gemm_launches, 1)
        alone_gbs = gemm_bytes / (gemm_alone_ms / 1e3) / 1e9 if gemm_alone_ms > 0 else None
        roof["cd_gemm"] = {
            "bound": "hbm", "unit": "GB/s", "peak": pk["hbm_gbs"],
            "achieved": per_launch / (avg_ms / 1e3) / 1e9,
            "kernel": "k_cd_gemm_tc", "launches": gemm_launches, "ms_total": gemm_ms,
            "bytes_per_launch": per_launch,
            "note": (f"k_cd_gemm_tc (tcgen05 exact-slice projections of the decomposition's "
                     f"streaming passes) in {args.steps} more steps of the same pipeline after "
                     f"the timed ones: {gemm_launches} launches, CUDA events around each on its "
                     f"stream (early returns of the steps that start no pass included); bytes "
                     f"per decomposition = nlive*(16*streamed + 260*(passes-1)) + 512*streamed "
                     f"({nlive} live pairs, {cd_stats['passes']} passes, {cd_stats['streamed']} "
                     f"vectors streamed)"),
            "nlive": nlive,
            "alone": {"achieved": alone_gbs, "ms_total": gemm_alone_ms,
                      "launches": gemm_alone_launches,
                      "frac": alone_gbs / pk["hbm_gbs"] if alone_gbs else None,
                      "note": "one cds_cd_decompose (tensor-core form) with no transform beside it, "
                              "the same events"},
            "cd_stats": cd_stats}
    elif fused:
        # one stage for both.  The decomposition is bound by FP32 instruction
        # issue (12 FP32 instructions per float-pair multiply-add in the
        # projections); the float-pair transform adds 11 per multiply-add on
        # the same pipes, the exact-slice transform runs on the tensor pipe
        N, o, nv = m.nbf, m.nocc, m.nbf - m.nocc
        tr_macs = float(M) * N * ((o + n_orb) * N + o * nv + n_orb * N)
        instr = (12.0 * 4 * cd_stats["streamed"] + 12.0 * cd_stats["extra"]) * npr
        if args.transform == "f32x2":
            instr += 11.0 * tr_macs
        med["cd_transform"] = med.pop("cd")
        med.pop("transform")
        roof.pop("cd")
        roof.pop("transform")
        roof["cd_transform"] = {
            "bound": "alu", "unit": "T FP32 instr/s", "peak": pk["fp32_issue_tinstr"],
            "achieved": instr / (med["cd_transform"] / 1e3) / 1e12,
            "note": (f"pipelined decomposition + transform (cds_cd_decompose_to_mo, transform "
                     f"{args.transform}): float-pair FMAs of the projections "
                     f"({cd_stats['passes']} streaming passes, {cd_stats['streamed']} vectors "
                     f"streamed)" + (" and of the transform GEMMs" if args.transform == "f32x2"
                                     else "; the transform's 21 slice-pair GEMMs run on the "
                                          "tensor pipe beside them") +
                     "; peak = 152 SMs x 128 FP32 lanes x 2.07 GHz"),
            "cd_stats": cd_stats}
    if fused and not gemm_timed:
        # the dominant kernels (k_cd_project_spec + k_cd_update, 62 % of the
        # step's launch list) timed alone: one float-pair decomposition on the
        # current stream, the one it launches on, bracketed by CUDA events
        cd_alone = []
        for _ in range(2):
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record()
            G.cds_cd_decompose(xyz, al, at, args.delta, args.scheme, L_out=Lbuf, workspace=cd_ws,
                               precision=args.cd_precision)
            a1.record()
            torch.cuda.synchronize()
            cd_alone.append(a0.elapsed_time(a1))
        t_cd = min(cd_alone)
        # the method's own work: the left-looking projections, npair M(M-1)/2
        # float-pair multiply-adds of 12 FP32 instructions each (the speculative
        # candidates' extra projections are not counted)
        cd_instr = 12.0 * npr * M * (M - 1) / 2.0
        spec_instr = (12.0 * G.cdsigma.cd_candidates() * cd_stats["streamed"] +
                      12.0 * cd_stats["extra"]) * npr
        roof["cd_kernels"] = {
            "bound": "alu", "unit": "T FP32 instr/s", "peak": pk["fp32_issue_tinstr"],
            "achieved": cd_instr / (t_cd / 1e3) / 1e12, "ms": t_cd,
            "issued_incl_speculation_tinstr_s": spec_instr / (t_cd / 1e3) / 1e12,
            "note": (f"k_cd_project_spec + k_cd_update (float-pair decomposition, M = {M}) timed "
                     f"alone after the timed steps (best of 2 calls) on the stream they launch "
                     f"on; achieved = the method's npair*M(M-1)/2 float-pair multiply-adds x 12 "
                     f"FP32 instructions / time ({cd_stats['passes']} streaming passes, "
                     f"{cd_stats['streamed']} vectors streamed, "
                     f"{G.cdsigma.cd_candidates()} candidates per pass); peak = 152 SMs x 128 "
                     f"FP32 lanes x 2.07 GHz (unit counts and the maximum clock, not measured)"),
            "cd_stats": cd_stats}
    for r in roof.values():
        r["frac"] = r["achieved"] / r["peak"]
        r["traffic"] = None
    if "cd_gemm" in roof:
        # DRAM bytes per algorithmic byte of k_cd_gemm_tc from one ncu capture
        # (the pass at k0 = 510 of the C60-shaped decomposition, 217,440 live
        # pairs, 512 columns: 1.837545 GB of dram__bytes_read + write against
        # 1.838065 GB), scaled to this run's average launch; traffic grows with
        # the columns streamed
        roof["cd_gemm"]["traffic"] = CD_GEMM_TRAFFIC_PER_BYTE * roof["cd_gemm"]["bytes_per_launch"]
    # (traffic stays null until an ncu capture of the current kernels exists)
    dominant = max(med, key=med.get)
    # the stage that dominates the step is the pipelined decomposition +
    # transform; the kernels that dominate it are the decomposition's
    dominant_roof = ("cd_gemm" if gemm_timed else "cd_kernels") if fused else dominant

    # ---- safeguarded Newton on the same numerators (quasiparticle roots) ----
    bracketed = None
    wb = None
    if cached:
        torch.cuda.synchronize()
        a0 = time.perf_counter()
        wb, Pb, itb, stb, brb = G.cds_qp_solve_bracketed_cached(cache, orbs, eps, m.nbf, m.nocc)
        torch.cuda.synchronize()
        bracketed = {"ms": (time.perf_counter() - a0) * 1e3,
                     "iters": itb.cpu().tolist(), "status": stb.cpu().tolist(),
                     "omega_Ha": wb.cpu().numpy().tolist(), "pole": Pb.cpu().numpy().tolist(),
                     "note": "Newton kept inside the pole-free interval around each e_q "
                             "(cds_qp_solve_bracketed_cached): the quasiparticle root of every "
                             "orbital; wall time incl. the host-side bracket"}

    # ---- the all-FP64 GPU step, measured once, and per-orbital accuracy ----
    fp64 = None
    if not args.no_fp64_arm and prec != "fp64":
        fp64 = run_fp64_step(args, m, xyz, al, at, C, eps, orbs, E, Lov, Lp, w, wb, value, pk)

    # ---- adjoint of the 8 orbitals around the gap (tensor cores) ----
    adjoint = None
    if not args.no_adjoint and prec != "fp64":
        adjoint = run_adjoint(m, Lov, Lp, orbs, eps, wb if wb is not None else w, pk)

    # ---- MP2 correlation energy (Eq. MP2) on the same factors ----
    mp2 = None
    if not args.no_mp2:
        mp2 = run_mp2(m, Lov, eps, prec if prec != "fp64" else "bf16x3", pk)

    # ---- the other transform form on the same vectors: time and error ----
    # (the split-product TF32X3 / BF16X3 forms refuse this C: its column
    # 1-norms reach 1.2e4, far beyond their FP32-accumulation bound)
    trtc = None
    if not args.no_trtc:
        trtc = {p_: run_transform_tc(m, L, C, orbs, Lov, p_)
                for p_ in ("f32x2", "ozaki") if not (fused and p_ == args.transform)}

    # ---- atomic Cholesky basis + V-approximation in place of the full CD ----
    acd = None
    if not args.no_acd:
        acd = run_acd(m, args.delta, orbs, eps, prec if prec != "fp64" else "bf16x3", w, P)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+" + prec, "data": "synthetic",
        "config": {"workload": WORKLOAD,
                   "delta": args.delta, "scheme": args.scheme, "cholesky_rank": M,
                   "orbitals": n_orb, "energies_per_orbital": m.nE, "newton_conv_Ha": 1e-5,
                   "precision": prec,
                   "transform_precision": args.transform if fused else tr_prec,
                   "newton": "cached numerators" if cached else "recomputed integrals",
                   "parallelism": f"replicas{dist.world}",
                   "l2": "inputs larger than L2 (L is %.1f GB, Lov %.0f MB)" % (M * npr * 8 / 1e9, Lov.numel() * 8 / 1e6)},
        "stages_ms": med,
        "qp": {"iters": iters.tolist(), "status": st.cpu().tolist(),
               "omega_Ha": w.cpu().numpy().tolist(), "pole": P.cpu().numpy().tolist()},
        "roofline": dict(roof[dominant_roof], kernel=dominant_roof, stage=dominant),
        "rooflines": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
        "peaks": pk,
        "fp64_step": fp64,
        "adjoint": adjoint,
        "mp2": mp2,
        "bracketed_newton": bracketed,
        "acd": acd,
        "transform_tc": trtc,
    }
    if not args.no_batched:
        result["batched"] = run_batched(args, device)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(m, M, iters)
    dist.done()
    return result


def run_fp64_step(args, m, xyz, al, at, C, eps, orbs, E, Lov_mx, Lp_mx, w_mx, wb_mx, value_mx,
                  pk):
    """One whole step of the method in FP64 on the GPU, timed stage by stage
    with CUDA events on the stream the calls launch on: FP64 decomposition
    (same delta and scheme), FP64 transform, the Sigma grid (64 energies) in
    FP64 keeping the FP64 numerators, and Newton from them (plain, as in the
    timed step; the safeguarded roots follow, untimed).  Per orbital, the
    quasiparticle energies of the split-precision forms (the timed step's
    BF16X3, and TF32X3 on the same factors) against these FP64 ones."""
    import torch
    import paper_0912_1459_gb300 as G

    n_orb = len(m.orbitals)
    dev = eps.device
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    torch.cuda.synchronize()
    ev[0].record()
    L, piv, D, de = G.cds_cd_decompose(xyz, al, at, args.delta, args.scheme, precision="fp64",
                                       max_rank=2048 if args.delta >= 1e-5 else 4096)
    ev[1].record()
    Lov, Lp = G.cds_cd_to_mo(L, C, m.nocc, orbs, precision="fp64")
    ev[2].record()
    sig, dsig, cache64 = G.cds_sigma2_diag_cache(Lov, Lp, eps, m.nocc, E, "fp64")
    ev[3].record()
    w, P, it, st = G.cds_qp_solve_cached(cache64, orbs, eps, m.nbf, m.nocc, conv=1e-5, max_iter=50,
                                         precision="fp64")
    ev[4].record()
    torch.cuda.synchronize()
    stages = {k: ev[i].elapsed_time(ev[i + 1])
              for i, k in enumerate(("cd", "transform", "sigma_grid", "qp"))}
    total_ms = sum(stages.values())
    wb, Pb, _, stb, _ = G.cds_qp_solve_bracketed_cached(cache64, orbs, eps, m.nbf, m.nocc,
                                                        precision="fp64")
    w64, P64, st64 = w.cpu().numpy(), P.cpu().numpy(), st.cpu().numpy()
    wb64 = wb.cpu().numpy()
    qp = (st64 == 0) & (P64 >= 0.5)
    mev = lambda x: (np.abs(x) * HARTREE_EV * 1e3).tolist()  # noqa: E731
    forms = {}
    # the timed step's own results (BF16X3 on its float-pair / exact-slice factors)
    e_plain = np.asarray(w_mx.cpu().numpy()) - w64
    forms[args.precision + " (timed step)"] = {
        "plain_newton_abs_err_meV": mev(e_plain),
        "max_over_qp_poles_meV": float(np.max(np.abs(e_plain[qp])) * HARTREE_EV * 1e3) if qp.any() else None,
        "bracketed_abs_err_meV": mev(wb_mx.cpu().numpy() - wb64) if wb_mx is not None else None}
    # TF32X3 on the same factors: Sigma grid keeping numerators, Newton from them
    for p2 in ("tf32x3",):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a0.record()
        _, _, cache2 = G.cds_sigma2_diag_cache(Lov_mx, Lp_mx, eps, m.nocc, E, p2)
        w2, P2, _, st2 = G.cds_qp_solve_cached(cache2, orbs, eps, m.nbf, m.nocc, conv=1e-5,
                                               max_iter=50, precision=p2)
        a1.record()
        torch.cuda.synchronize()
        wb2 = G.cds_qp_solve_bracketed_cached(cache2, orbs, eps, m.nbf, m.nocc, precision=p2)[0]
        e2 = w2.cpu().numpy() - w64
        forms[p2] = {"sigma_grid_plus_newton_ms": a0.elapsed_time(a1),
                     "plain_newton_abs_err_meV": mev(e2),
                     "max_over_qp_poles_meV": float(np.max(np.abs(e2[qp])) * HARTREE_EV * 1e3) if qp.any() else None,
                     "bracketed_abs_err_meV": mev(wb2.cpu().numpy() - wb64)}
        del cache2
    del cache64
    v64 = n_orb / (total_ms / 1e3)
    return {"stages_ms": stages, "ms": total_ms, "solves_per_s": v64,
            "mixed_over_fp64": value_mx / v64, "cholesky_rank": int(L.shape[0]),
            "orbitals": [int(q) for q in m.orbitals], "fp64_pole": P64.tolist(),
            "fp64_status": st64.tolist(), "fp64_bracketed_status": stb.cpu().tolist(),
            "qp_poles": int(qp.sum()), "forms": forms,
            "note": "measured once after the timed steps: FP64 CD + FP64 transform + FP64 Sigma "
                    "grid (64 energies, numerators kept) + FP64 Newton from them; errors per "
                    "orbital against it, plain Newton (Eq. iter) and safeguarded roots; "
                    "max_over_qp_poles covers the orbitals whose FP64 root has P >= 0.5"}


def run_adjoint(m, Lov, Lp, orbs, eps, omega, pk, reps: int = 3):
    """The hand-written adjoint (cds_qp_gradient, BF16X3 tensor cores) for the
    8 orbitals around the gap (HOMO-3 .. LUMO+3) at the given roots: CUDA-event
    time of one call after a warm-up, and the rate of its tensor work."""
    import torch
    import paper_0912_1459_gb300 as G

    n_orb = len(m.orbitals)
    mid = n_orb // 2
    sel = torch.arange(mid - 4, mid + 4, device=Lp.device)
    Lp8 = Lp[sel].contiguous()
    o8, w8 = orbs[sel].contiguous(), omega[sel].contiguous()
    g = torch.ones(8, dtype=torch.float64, device=Lp.device)
    G.cdsigma.cds_qp_gradient(Lov, Lp8, o8, eps, m.nocc, w8, g, "bf16x3")
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        G.cdsigma.cds_qp_gradient(Lov, Lp8, o8, eps, m.nocc, w8, g, "bf16x3")
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    o, v, M = Lov.shape
    # per orbital: X (both sums), dLq and dLov GEMMs, each 2 M (o v)(o + v) MACs-as-flops,
    # 3 split products
    flops = 8 * 3 * 3 * 2.0 * M * (o * v) * (o + v)
    ach = flops / (t / 1e3) / 1e12
    return {"orbitals": [int(q) for q in o8.cpu().tolist()], "precision": "bf16x3", "ms": t,
            "roofline": {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach,
                         "peak": pk["bf16_tflops"], "frac": ach / pk["bf16_tflops"],
                         "note": "3 GEMMs per orbital (X, dLq, dLov), 2 M (o v)(o+v) flops each, "
                                 "x 3 split products; of measured burst BF16 peak"},
            "note": "d(eps, Lov, Lp) of sum_t w_t at the safeguarded roots; the G pass, "
                    "splits and transposes included in the time"}


def run_mp2(m, Lov, eps, prec, pk, reps: int = 3):
    """Eq. MP2 on the step's factors: CUDA-event time of cds_mp2_energy (after
    one untimed call that also sizes the workspace), the rate of its tensor
    work, and the energy."""
    import torch
    import paper_0912_1459_gb300 as G

    o, v, M = Lov.shape
    lib = G.load()
    ws = torch.empty(lib.cds_mp2_workspace_bytes(o + v, o, M, G.cdsigma.PRECISIONS[prec]),
                     dtype=torch.uint8, device=Lov.device)
    tot, _ = G.cds_mp2_energy(Lov, eps, o, prec, workspace=ws)
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        tot, _ = G.cds_mp2_energy(Lov, eps, o, prec, workspace=ws)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    # the kernel forms every (ia|jb) for all ordered (i, j): 2 M (o v)^2, x3 split products
    flops = 3 * 2.0 * M * (o * v) ** 2
    ach = flops / (t / 1e3) / 1e12
    return {"precision": prec, "ms": t, "e_corr_Ha": float(tot),
            "roofline": {"bound": "tensor", "unit": "TFLOP/s", "achieved": ach,
                         "peak": pk["bf16_tflops"], "frac": ach / pk["bf16_tflops"],
                         "note": "3 split products x 2 M (o v)^2 per evaluation"}}


def run_transform_tc(m, L, C, orbs, Lov_ref, prec):
    """One transform form on the step's Cholesky vectors: CUDA-event time of
    one call after a warm-up, and its error against the step's Lov.  TF32X3
    accumulates in FP32 and cannot carry the cancellation of this C (|C| up
    to 106); the exact-slice form (ozaki) and float pairs can."""
    import torch
    import paper_0912_1459_gb300 as G

    lib = G.load()
    M = L.shape[0]
    ws = torch.empty(lib.cds_cd_to_mo_workspace_bytes(m.nbf, m.nbf, m.nocc, M, len(m.orbitals)),
                     dtype=torch.uint8, device=L.device)
    G.cds_cd_to_mo(L[:32], C, m.nocc, orbs, workspace=ws, precision=prec)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    Lov, _ = G.cds_cd_to_mo(L, C, m.nocc, orbs, workspace=ws, precision=prec)
    b.record()
    torch.cuda.synchronize()
    t = a.elapsed_time(b)
    err = float((Lov - Lov_ref).abs().max() / Lov_ref.abs().max())
    # products per multiply-add: 3 split (tf32x3), 21 slice pairs (ozaki), 1 (f32x2)
    N, o, v, np_ = m.nbf, m.nocc, m.nbf - m.nocc, len(m.orbitals)
    macs = float(M) * ((o + np_) * N * N + o * v * N + np_ * N * N)
    prods = {"tf32x3": 3, "ozaki": 21, "f32x2": 1}[prec]
    return {"ms": t, "tflops_of_products": prods * 2.0 * macs / (t / 1e3) / 1e12,
            "lov_rel_err_vs_step": err}


def run_acd(m, delta, orbs, eps, prec, w_cd, P_cd):
    """Sec. II.A atomic CD with the V-approximation (Eq. int_approx) in place of
    the full decomposition: CUDA-event times of the basis choice and of the
    factors B, the float-pair transform of B, the Newton solve on it, and the
    quasiparticle energies' difference from the full-CD step (poles >= 0.5)."""
    import torch
    import paper_0912_1459_gb300 as G

    dev = eps.device
    xyz = torch.from_numpy(m.basis.xyz).to(dev)
    al = torch.from_numpy(m.basis.alpha).to(dev)
    at = torch.from_numpy(m.basis.atom.astype(np.int32)).to(dev)
    C = torch.from_numpy(m.C).to(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    G.cds_ri_factors(xyz, al, G.cds_acd_aux_pairs(al, at, delta)[:8], "f32x2")   # warm-up
    torch.cuda.synchronize()
    ev[0].record()
    aux = G.cds_acd_aux_pairs(al, at, delta)
    ev[1].record()
    B = G.cds_ri_factors(xyz, al, aux, "f32x2")
    ev[2].record()
    Lov, Lp = G.cds_cd_to_mo(B, C, m.nocc, orbs, precision="f32x2")
    ev[3].record()
    w, P, it, st = G.cds_qp_solve(Lov, Lp, orbs, eps, m.nocc, precision=prec)
    ev[4].record()
    torch.cuda.synchronize()
    t = [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]
    qp = ((P_cd >= 0.5) & (st == 0)).cpu().numpy()
    diff = np.abs((w - w_cd).cpu().numpy()) * HARTREE_EV * 1e3
    return {"naux": int(aux.numel()), "basis_ms": t[0], "factors_ms": t[1], "transform_ms": t[2],
            "qp_ms": t[3], "status": st.cpu().tolist(),
            "qp_vs_full_cd_meV": diff[qp].tolist(),
            "note": "one-centre basis densities of the isolated atoms' CD at the same delta; "
                    "B = L_m^-1 (rho~|rho) on the GPU (float pairs), then the step's transform "
                    "and Newton (recomputing form); times of one call each after a warm-up"}


# ----------------------------------------------------------------------------
# batched workload: 64 clusters in one pipeline, Sigma/Newton under a graph
# ----------------------------------------------------------------------------
def run_batched(args, device):
    """Batched clusters (centre counts U{4..40}, 10 s-Gaussians per centre,
    o = N/5, delta = 1e-5, U{4..16} orbitals on U{8..64} energies): batch CD,
    transform, then the Sigma-grid + Newton stage as an autotuned CUDA graph.
    Reports aggregate solves/s of the graph and per-cluster latency from the
    device-side completion stamps."""
    import torch
    from paper_0912_1459_gb300 import autotune
    from paper_0912_1459_gb300 import cdsigma as C

    mols = W.config3()
    spec = [(mm.nbf, mm.nocc, len(mm.orbitals), mm.nE, C.default_max_rank(mm.nbf)) for mm in mols]
    cdp = "fp64" if args.precision == "fp64" else args.cd_precision
    b = C.Batch(spec, device, "bf16x3" if args.precision == "fp64" else args.precision,
                cd_precision=cdp)
    cat = lambda xs: torch.from_numpy(np.ascontiguousarray(np.concatenate(xs))).to(device)  # noqa: E731
    xyz = cat([mm.basis.xyz.ravel() for mm in mols])
    al = cat([mm.basis.alpha for mm in mols])
    at = cat([mm.basis.atom.astype(np.int32) for mm in mols])
    Cc = cat([mm.C.ravel() for mm in mols])
    eps = cat([mm.eps for mm in mols])
    orb = cat([mm.orbitals.astype(np.int32) for mm in mols])
    E = cat([W.energy_grid(mm.eps[mm.orbitals], mm.nE).ravel() for mm in mols])
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    M = b.cd_decompose(xyz, al, at, 1e-5, precision=cdp)
    ev[1].record()
    b.cd_to_mo(Cc, orb, precision=args.transform if args.precision != "fp64" else "fp64")
    ev[2].record()
    torch.cuda.synchronize()
    tuned = autotune.tune(b, orb, eps, E)
    g = b.graph(orb, eps, E)
    g.launch()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 3)
    t0.record()
    for _ in range(reps):
        g.launch()
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    st = b.stamps.cpu().numpy().astype(np.float64)
    lat_ms = (st[1:] - st[0]) / 1e6
    n_solves = int(sum(len(mm.orbitals) for mm in mols))
    status = b.status[:n_solves].cpu().numpy()
    cd_ms, tr_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    whole_ms = cd_ms + tr_ms + ms
    return {"clusters": len(mols), "nbf_range": [int(min(x[0] for x in spec)), int(max(x[0] for x in spec))],
            "solves": n_solves, "energies": int(sum(x[2] * x[3] for x in spec)),
            "cd_ms": cd_ms, "transform_ms": tr_ms,
            "whole_ms": whole_ms, "whole_solves_per_s": n_solves / (whole_ms / 1e3),
            "cd_precision": cdp,
            "transform_precision": args.transform if args.precision != "fp64" else "fp64",
            "graph_ms": ms, "solves_per_s": n_solves / (ms / 1e3),
            "latency_ms_p50": float(np.percentile(lat_ms, 50)),
            "latency_ms_p99": float(np.percentile(lat_ms, 99)),
            "converged": int((status == 0).sum()), "ranks": [int(x) for x in M],
            "autotune": {"choice": list(tuned["choice"]), "ms": tuned["ms"], "cached": tuned["cached"]},
            "note": "whole = batched decomposition + transform + one graph replay (every "
                    "cluster from its basis to its roots); graph = Sigma on every cluster's "
                    "energy grid + Newton (50 passes max) in one replay, solves_per_s counts "
                    "the graph alone; latency = device stamp of a cluster's last retired orbital "
                    "minus the replay's start stamp"}


# ----------------------------------------------------------------------------
# CPU oracle legs (the only place bench.py runs oracle/)
# ----------------------------------------------------------------------------
def oracle_sample(m, M_full: int, iters_per_orbital: float, n_cd=(24, 48), n_tr=4):
    """Time the oracle on a bounded sample and scale to one full step.

    CD: the first n_cd[0] and n_cd[1] Gram-Schmidt steps on the real basis,
    fitted by t(k) = a k + b k^2 / 2 (ERI column + projections) and evaluated
    at M; transform: n_tr vectors, scaled linearly to M; self-energy: one orbital on
    synthetic factors of the full shape at 1 and 2 energies (GEMM + per-energy
    epilogue), scaled to 20 orbitals x (64 energies + Newton passes)."""
    from oracle import ao2mo, cd, eri, sigma2

    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    times = []
    for k in n_cd:
        a = time.perf_counter()
        try:
            cd.decompose(pd, 1e-300, max_rank=k)
        except cd.RankCapError:
            pass
        times.append(time.perf_counter() - a)
        if k == n_cd[-1]:
            break
    (k1, k2), (t1, t2) = n_cd, times
    # t = a k + b k^2/2  (two equations)
    b = (t2 / k2 - t1 / k1) * 2.0 / (k2 - k1)
    a_ = t1 / k1 - b * k1 / 2.0
    t_cd = a_ * M_full + b * M_full ** 2 / 2.0
    rng = np.random.default_rng(0)
    Lsmall = rng.standard_normal((n_tr, pd.npair)) * 1e-2
    a = time.perf_counter()
    ao2mo.mo_factors(Lsmall, m.C, m.nocc, m.orbitals)
    t_tr = (time.perf_counter() - a) * M_full / n_tr
    o, v = m.nocc, m.nbf - m.nocc
    Lov = rng.standard_normal((o, v, M_full)) * 1e-2
    Lq = rng.standard_normal((m.nbf, M_full)) * 1e-2
    q = int(m.orbitals[len(m.orbitals) // 2])
    a = time.perf_counter()
    sigma2.sigma2_from_factors(Lq, Lov, m.eps, m.nocc, [m.eps[q]])
    s1 = time.perf_counter() - a
    a = time.perf_counter()
    sigma2.sigma2_from_factors(Lq, Lov, m.eps, m.nocc, [m.eps[q], m.eps[q] + 0.01])
    s2 = time.perf_counter() - a
    per_e = max(s2 - s1, 0.0)
    n_orb = len(m.orbitals)
    t_grid = n_orb * (s1 + (m.nE - 1) * per_e)
    t_qp = n_orb * iters_per_orbital * s1
    total = t_cd + t_tr + t_grid + t_qp
    wall = sum(times) + t_tr * n_tr / M_full + s1 + s2
    return {"value": n_orb / total, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": (f"oracle (numpy FP64) timed on CD steps {n_cd}, {n_tr} transform vectors and "
                       f"one orbital's Sigma at 1 and 2 energies (full shape); scaled to one step "
                       f"(M={M_full}, 20 orbitals x 64 energies + {iters_per_orbital:.1f} Newton "
                       f"passes/orbital): CD {t_cd:.1f}s transform {t_tr:.1f}s Sigma grid "
                       f"{t_grid:.1f}s Newton {t_qp:.1f}s"),
            "sample_wall_s": wall,
            "stage_s_estimate": {"cd": t_cd, "transform": t_tr, "sigma_grid": t_grid, "qp": t_qp}}


# One sample size for both oracle legs (cpu_baseline here, the reference arm's
# steps), so that they model the same step from the same measurements.
ORACLE_SAMPLE = {"n_cd": (32, 64), "n_tr": 4}


def cpu_baseline(m, M, iters):
    # ~10-20 s of oracle work on the host cores
    return oracle_sample(m, M, float(np.mean(iters)), **ORACLE_SAMPLE)


def run_reference(args, dist: Dist):
    """The CPU oracle as the reference arm: rank 0 only, bounded samples."""
    if dist.world > 1 and dist.rank != 0:
        return None
    m, _ = workload(args.delta)
    M_full = {1e-3: 510, 1e-4: 896, 1e-5: 1436}.get(args.delta, 896)
    iters = 4.0
    for _ in range(args.warmup):
        oracle_sample(m, M_full, iters, n_cd=(4, 8), n_tr=1)
    vals, walls = [], []
    for _ in range(args.steps):
        s = oracle_sample(m, M_full, iters, **ORACLE_SAMPLE)
        vals.append(s["value"])
        walls.append(s["sample_wall_s"])
    value = float(np.median(vals))
    cb = {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
          "sample": s["sample"] + f"; sample wall time {np.median(walls):.1f} s per step"}
    # ms_per_step: the modelled time of one whole step (20 solves / value),
    # not the wall time of the bounded sample
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 20.0 / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "delta": args.delta, "scheme": args.scheme,
                       "cholesky_rank": M_full, "orbitals": 20, "energies_per_orbital": 64,
                       "newton_conv_Ha": 1e-5, "precision": "fp64", "transform_precision": "fp64",
                       "parallelism": "cpu-oracle"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        res = run_reference(args, dist)
    else:
        res = run_ours(args, dist)
    if res is not None and dist.rank == 0:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
