"""Writes oracle golden files for the workloads too large to recompute inside a test run.

Only the CPU oracle (``oracle/``) and the seeded input generators (``synth/``) are used.  Usage:

    python tests/golden/make_golden.py rmat20_wc      # R-MAT scale 20, weighted cascade, R=256, K=50

Output: ``tests/golden/<name>.json`` with, for the first diffusion, the SHA-256 of the n*R register bytes, sweeps,
edge-simulation visits and the frontier sizes, and for the whole seed selection the per-step seeds, sigma, estimate,
register sums and rebuild flags plus the run totals.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from synth import workloads  # noqa: E402


def run(name: str) -> dict:
    prob = getattr(workloads, name)()
    g = prob.graph
    out = dict(workload=prob.name, n=g.n, m=g.m, model=prob.model, p=prob.p, R=prob.R, K=prob.K, eps_g=prob.eps_g,
               eps_l=prob.eps_l, eps_c=prob.eps_c, seed=prob.seed)
    t = time.time()
    M, sweeps, visits, log = oracle.build_sketch(g.n, g.xadj, g.adj, prob.model, prob.p, prob.R, prob.seed,
                                                 eps_c=prob.eps_c)
    out["build"] = dict(sha256=hashlib.sha256(M.tobytes()).hexdigest(), sweeps=sweeps, visits=visits,
                        frontier=[int(x) for x in log], seconds=time.time() - t)
    del M
    print(f"build done in {out['build']['seconds']:.1f}s: {sweeps} sweeps, {visits} visits", flush=True)
    t = time.time()
    r = oracle.select_seeds(g.n, g.xadj, g.adj, prob.model, prob.p, prob.R, prob.K, prob.eps_g, prob.eps_l,
                            prob.eps_c, prob.seed)
    out["select"] = dict(seeds=[int(x) for x in r["seeds"]], sigma=[float(x) for x in r["sigma"]],
                         estimate=[float(x) for x in r["est"]], gsum=[int(x) for x in r["gsum"]],
                         rebuilt=[int(x) for x in r["rebuilt"]], visits=r["visits"], sweeps=r["sweeps"],
                         builds=r["builds"], seconds=time.time() - t)
    print(f"select done in {out['select']['seconds']:.1f}s", flush=True)
    return out


if __name__ == "__main__":
    for name in sys.argv[1:]:
        res = run(name)
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(res, f, indent=1)
