"""Write tests/golden/batch_oracle.json: the CPU oracle's results for a
subsample of the 256-instance batched mix (paper_1903_11554_gb300.inputs.
batched_mix(256)): the 24 instances with the smallest d * sum(N_k) * cap^2 (so
the oracle finishes in minutes), keyed by their index in the mix: each run's
value, status and final ranks, the 60-digit contraction of its final cores,
the FP64 value's own error against it, and the tolerance a GPU value is held
to (ten times that error, at least 1e-12).  Calls only the oracle.

    python tests/golden/make_batch_values.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ttcross  # noqa: E402
from paper_1903_11554_gb300 import inputs  # noqa: E402


def subsample(probs, count=24):
    cost = sorted((p.d * sum(p.N) * p.rank_cap ** 2, i) for i, p in enumerate(probs))
    return sorted(i for _, i in cost[:count])


def main():
    probs = inputs.batched_mix(256)
    out = {}
    for i in subsample(probs):
        p = probs[i]
        t = time.time()
        r = ttcross.integrate(p)
        st = r["state"]
        exact = ttcross.contract_decimal(p, st, [ttcross.core(p, st, k) for k in range(1, p.d + 1)])
        fp64_err = abs(r["value"] - exact) / abs(exact)
        out[str(i)] = {"workload": p.name, "value": repr(r["value"]), "status": r["status"], "sweeps": r["sweeps"],
                       "n_eval": r["n_eval"], "ranks": r["ranks"], "value_exact_contraction": repr(exact),
                       "oracle_fp64_rel_err": fp64_err,
                       # an FP64 contraction of this cross is good to about the oracle's own error:
                       # ten times it, and at least 1e-12
                       "tolerance": max(1e-12, 10.0 * fp64_err),
                       "oracle_seconds": round(time.time() - t, 1)}
        print(i, out[str(i)], flush=True)
    json.dump(out, open(os.path.join(HERE, "batch_oracle.json"), "w"), indent=1)


if __name__ == "__main__":
    main()
