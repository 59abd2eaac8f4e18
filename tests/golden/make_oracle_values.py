"""Write tests/golden/oracle_full.json: the CPU oracle's results on the full
C_4, D_12 and E_16 workloads (seeded, synthetic grids from
paper_1903_11554_gb300.inputs).  Calls only the oracle; takes ~15 min.

    python tests/golden/make_oracle_values.py [c4 d12 e16]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ttcross  # noqa: E402
from paper_1903_11554_gb300 import inputs  # noqa: E402

CONFIGS = {"c4": inputs.config_c4, "d12": inputs.config_d12, "e16": inputs.config_e16}


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
            "parents": {k: [list(map(int, a)) for a in v] for k, v in par.items()},
            "oracle_seconds": round(time.time() - t, 1),
        }
        json.dump(out, open(path, "w"), indent=1)
        print(name, out[name]["value"], out[name]["sweeps"], out[name]["oracle_seconds"], "s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c4", "d12", "e16"])
