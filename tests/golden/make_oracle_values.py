"""Write tests/golden/oracle_full.json: the CPU oracle's results on the full
C_4, D_12 and E_16 workloads and on D_8 and D_16 in the paper's unit-cube form
with Gauss-Legendre 129 nodes and C_8 .. C_32 in that form with 33 nodes (seeded, synthetic grids from
paper_1903_11554_gb300.inputs): value, status, sweeps, evaluations, final
ranks and nested sets, per sweep the integral and the ranks, and the final
cross contracted at 60 digits (oracle.ttcross.contract_decimal).  Calls only
the oracle; takes ~40 min.

    python tests/golden/make_oracle_values.py [c4 d12 d12_r4 d12_p4 e16 d8 d16 c8_cube c16_cube c24_cube c32_cube]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ttcross  # noqa: E402
from paper_1903_11554_gb300 import inputs  # noqa: E402

CONFIGS = {"c4": inputs.config_c4, "d12": inputs.config_d12, "d12_r4": inputs.config_d12_r4,
           "d12_p4": inputs.config_d12_p4,
           "e16": inputs.config_e16,
           "d8": lambda: inputs.config_d_cube(8), "d16": lambda: inputs.config_d_cube(16),
           "c8_cube": lambda: inputs.config_c_cube(8), "c16_cube": lambda: inputs.config_c_cube(16),
           "c24_cube": lambda: inputs.config_c_cube(24), "c32_cube": lambda: inputs.config_c_cube(32)}


def main(names):
    path = os.path.join(HERE, "oracle_full.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        p = CONFIGS[name]()
        t = time.time()
        r = ttcross.integrate(p)
        st = r["state"]
        par = ttcross.to_parents(p, st)
        out[name] = {
            "workload": p.name,
            "value": repr(r["value"]),
            "status": r["status"],
            "sweeps": r["sweeps"],
            "n_eval": r["n_eval"],
            "ranks": r["ranks"],
            "internal_conv": r["internal_conv"],
            "history": [repr(h.value) for h in r["history"]],
            "history_ranks": [list(map(int, h.ranks)) for h in r["history"]],
            # the same final cross contracted at 60 digits (Sec. 4.1's product of
            # the oracle's FP64 cores): what the FP64 value above rounds
            "value_exact_contraction": repr(ttcross.contract_decimal(
                p, st, [ttcross.core(p, st, k) for k in range(1, p.d + 1)])),
            "parents": {k: [list(map(int, a)) for a in v] for k, v in par.items()},
            "oracle_seconds": round(time.time() - t, 1),
        }
        json.dump(out, open(path, "w"), indent=1)
        print(name, out[name]["value"], out[name]["sweeps"], out[name]["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CONFIGS))
