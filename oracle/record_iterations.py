"""Record the oracle's iteration count per benchmark workload.

Test infrastructure: runs only the seeded input generator and the FP64 CPU
oracle (no library code), and writes oracle/iterations.json, which the
benchmark's CPU-baseline leg uses to turn a bounded sample of oracle
iterations into solves per second.

    python oracle/record_iterations.py
"""
from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import gridgen  # noqa: E402
import oracle  # noqa: E402

# name: (grid, configuration index for the seed, pattern, drop tolerance, band q, rtol)
WORKLOADS = {
    "orca12-fp64": (gridgen.ORCA12, 4, oracle.PAT_TRIL_A2, 0.05, 0, 1e-10),
    "orca12-fp64-trilA": (gridgen.ORCA12, 4, oracle.PAT_TRIL_A, 0.0, 0, 1e-10),
    "orca025-fp64": (gridgen.ORCA025, 2, oracle.PAT_TRIL_A2, 0.05, 0, 1e-10),
    "coarse-fp64": (gridgen.COARSE, 1, oracle.PAT_TRIL_A2, 0.05, 0, 1e-10),
}


def main():
    out = {}
    for name, (cfg, ci, pat, tau, q, rtol) in WORKLOADS.items():
        t = time.time()
        g = gridgen.make_grid(seed=gridgen.seed_for(ci), **cfg)
        P = oracle.OracleProblem.from_grid(g)
        assert P.ainv(pat, tau, q) == oracle.OK
        r = P.pcg(P.to_wet(g.b), rtol=rtol)
        assert r.status == oracle.OK, r.status
        out[name] = r.iters
        print(f"{name}: {r.iters} iterations, true relres {r.true_relres:.2e} ({time.time() - t:.0f} s)", flush=True)
    with open(os.path.join(ROOT, "oracle", "iterations.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
