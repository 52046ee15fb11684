"""Write tests/golden/bench_golden.json: the CPU oracle's complete result on the
full-size workloads that bench.py times (and the n=4096 peer workload).

Calls only the oracle (plain C, Algorithms 2-4) and the seeded input
generators; nothing here touches the CUDA library.  Run from the repository
root:  python tests/golden/make_bench_golden.py
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1106_5694_gb300 import inputs  # noqa: E402

WORKLOADS = [
    {"name": "peer_n4096_seed0", "generator": "peer_shaped", "n": 4096, "seed": 0},
    {"name": "peer_n10000_seed0", "generator": "peer_shaped", "n": 10000, "seed": 0},
]


def sha(arr) -> str:
    return hashlib.sha256(np.ascontiguousarray(arr).tobytes()).hexdigest()


def main():
    out = {"_source": "oracle.dgs_parallel (plain C, Algorithms 2-4 with readings R1-R5), greedy start; "
                      "written by tests/golden/make_bench_golden.py", "workloads": []}
    for w in WORKLOADS:
        a = getattr(inputs, w["generator"])(w["n"], w["seed"])
        t0 = time.time()
        r = oracle.dgs_parallel(a)
        dt = time.time() - t0
        g = oracle.greedy_init(a)
        rec = dict(w)
        rec.update({"a_sha256": sha(a), "status": int(r.status), "objective": int(r.objective),
                    "sweeps": int(r.sweeps), "swaps_applied": int(r.swaps_applied),
                    "tau_sha256": sha(r.tau.astype(np.int32)),
                    "greedy_objective": int(oracle.objective(a, g)), "greedy_tau_sha256": sha(g.astype(np.int32)),
                    "oracle_seconds": round(dt, 1)})
        out["workloads"].append(rec)
        print(rec, flush=True)
    with open(os.path.join(ROOT, "tests", "golden", "bench_golden.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
