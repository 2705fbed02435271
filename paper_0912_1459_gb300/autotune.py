"""Autotuner for the batched tensor-core self-energy.

Times captured-graph replays of the actual batch for the library's kernel
configurations -- energies per epilogue pass of the tensor-core kernel
(8 / 16), work-item order (interleaved / blocked), the register tile of the
kernel that evaluates the grid from the kept numerators (2 / 4 / 8 energies
per pass) and how the Newton passes evaluate Sigma (streaming the kept
numerators; one candidate recomputes the integrals on the tensor cores) --
keeps the fastest, and caches the choice in a JSON file keyed by the batch's
shape signature (molecule sizes, orbital and energy counts, Cholesky ranks,
precision), so a repeated batch shape is tuned once.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

import torch

from . import cdsigma as C

# (energy chunk, item order, Newton from kept numerators, grid energies per pass)
CANDIDATES = ([(c, o, 1, ec) for c in (16, 8) for o in (0, 1) for ec in (4, 8, 2)] +
              [(16, 0, 0, 4)])


def cache_path() -> str:
    return os.environ.get("CDS_AUTOTUNE_CACHE",
                          os.path.join(tempfile.gettempdir(), "cdsigma_autotune.json"))


def signature(batch: "C.Batch") -> str:
    spec = [(m.nbf, m.nocc, m.np, m.nE, r) for m, r in zip(batch.mols, batch.M)]
    return hashlib.sha1(json.dumps([batch.prec, spec]).encode()).hexdigest()[:16]


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache: dict) -> None:
    path = cache_path()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)


def apply(choice) -> None:
    C.cds_tune_set(C.TUNE_ENERGY_CHUNK, int(choice[0]))
    C.cds_tune_set(C.TUNE_ITEM_ORDER, int(choice[1]))
    C.cds_tune_set(C.TUNE_NEWTON_CACHE, int(choice[2]))
    C.cds_tune_set(C.TUNE_GRID_EC, int(choice[3]) if len(choice) > 3 else 4)


def tune(batch: "C.Batch", orb, eps, E, reps: int = 2, use_cache: bool = True) -> dict:
    """Pick and apply the fastest configuration for this batch.

    Returns {"choice": (chunk, order, cache, grid_ec), "ms": {candidate: ms}, "cached": bool}."""
    key = "v3:" + signature(batch)
    cache = _load() if use_cache else {}
    if key in cache:
        choice = tuple(cache[key]["choice"])
        apply(choice)
        return {"choice": choice, "ms": cache[key]["ms"], "cached": True}
    timings = {}
    for cand in CANDIDATES:
        apply(cand)
        g = batch.graph(orb, eps, E)
        g.launch()                              # warm-up replay
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            g.launch()
        t1.record()
        torch.cuda.synchronize()
        timings[",".join(str(x) for x in cand)] = t0.elapsed_time(t1) / reps
        del g
    best = min(timings, key=timings.get)
    choice = tuple(int(x) for x in best.split(","))
    apply(choice)
    if use_cache:
        cache[key] = {"choice": list(choice), "ms": timings}
        _store(cache)
    return {"choice": choice, "ms": timings, "cached": False}
