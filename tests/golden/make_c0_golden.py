"""Writes c0_oracle.json: the oracle's results on the tiny 24-function case.

Only workloads/ (seeded inputs) and oracle/ are used.  The stored values are a
regression pin for the oracle (tests/test_golden.py re-derives them) and the
expected values of the GPU path on the same inputs.

    python tests/golden/make_c0_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import ao2mo, cd, eri, qp, sigma2  # noqa: E402


def compute() -> dict:
    m = W.config0()
    pd = eri.PairData(m.basis.xyz, m.basis.alpha)
    out = {"case": "tiny-N24 (6 centres, 4 s-Gaussians each, o = 6), seed 0",
           "delta": m.delta}
    res = cd.decompose(pd, m.delta)
    out["cd"] = {"M": int(res.M), "delta_eff": float(res.delta_eff),
                 "piv": [int(p) for p in res.piv],
                 "max_residual": float(res.D.max())}
    Lov, Lp = ao2mo.mo_factors(res.L, m.C, m.nocc, m.orbitals)
    out["orbitals"] = [int(q) for q in m.orbitals]
    sig, dsig = [], []
    for t, q in enumerate(m.orbitals):
        s, d = sigma2.sigma2_from_factors(Lp[t], Lov, m.eps, m.nocc, [m.eps[q]])
        sig.append(float(s[0]))
        dsig.append(float(d[0]))
    out["sigma_at_eps"] = sig
    out["dsigma_at_eps"] = dsig
    qps = []
    for t, q in enumerate(m.orbitals):
        def f(w, t=t):
            s, d = sigma2.sigma2_from_factors(Lp[t], Lov, m.eps, m.nocc, [w])
            return s[0], d[0]
        w, P, it, st = qp.newton_qp(f, m.eps[q], conv=1e-5, max_iter=50)
        qps.append({"omega": float(w), "pole": float(P), "iters": int(it), "status": int(st)})
    out["qp"] = qps
    return out


def main() -> None:
    path = os.path.join(HERE, "c0_oracle.json")
    out = compute()
    with open(path, "w") as f:   # one key per line, values compact
        f.write("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}" for k, v in out.items())
                + "\n}\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
