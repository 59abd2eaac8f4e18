"""Write tests/golden/c_grid_exact.json: for C_n in R^n on the trapezoid grid
of paper_1903_11554_gb300.inputs.config_c_rn_grid (n = 8, 16), the
exact tensor-product sum of the grid (oracle/exact.py: the separable 1-D
integral of the C integrand at 40 digits) and the CPU oracle's TT-cross run on
the same problem.  The tolerance stored for the GPU test is ten times the
oracle's own error against the exact grid value, and at least 5e-12.  Calls
only the oracle; needs mpmath; takes ~20 min.

    python tests/golden/make_c_grid_values.py [8 16]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact, integrands, ttcross  # noqa: E402
from paper_1903_11554_gb300 import inputs  # noqa: E402


def main(ns):
    path = os.path.join(HERE, "c_grid_exact.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for n in ns:
        p = inputs.config_c_rn_grid(n)
        t = time.time()
        grid = integrands.family_constant("C", "rn", n) * exact.c_grid_exact(p.nodes, p.weights)
        r = ttcross.integrate(p)
        err = abs(r["value"] / grid - 1)
        out[str(n)] = {"workload": p.name, "value": repr(grid), "oracle_value": repr(r["value"]),
                       "oracle_rel_err": err, "oracle_status": r["status"], "oracle_max_rank": r["max_rank"],
                       "tolerance": max(5e-12, 10.0 * err), "seconds": round(time.time() - t, 1)}
        json.dump(out, open(path, "w"), indent=1)
        print(n, out[str(n)], flush=True)


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [8, 16])
