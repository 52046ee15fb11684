"""Write tests/golden/bench_golden.json: the CPU oracle's complete result on the
full-size single-instance workloads (peer-shaped and uniform [0, 1e6), n =
4096, 10000 and 20000), and for uniform n = 20000 also a 50-sweep prefix.

Calls only the oracle (plain C, Algorithms 2-4) and the seeded input
generators; nothing here touches the CUDA library.  The oracle's slot
evaluations run on several host threads reading columns from a transposed
copy (oracle.set_evaluation); the oracle pins check that this gives the
literal single-threaded solve exactly.  Run from the repository root:

    python tests/golden/make_bench_golden.py [workload names ...] [--threads T]

With no names every workload is (re)written; existing records of other
workloads are kept.
"""
import argparse
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

PATH = os.path.join(ROOT, "tests", "golden", "bench_golden.json")
PREFIX_SWEEPS = 50

WORKLOADS = [
    {"name": "peer_n4096_seed0", "generator": "peer_shaped", "n": 4096, "seed": 0},
    {"name": "peer_n10000_seed0", "generator": "peer_shaped", "n": 10000, "seed": 0},
    {"name": "uniform_n4096_seed0", "generator": "uniform", "n": 4096, "seed": 0, "lo": 0, "hi": 10**6},
    {"name": "peer_n20000_seed0", "generator": "peer_shaped", "n": 20000, "seed": 0},
    {"name": "uniform_n10000_seed0", "generator": "uniform", "n": 10000, "seed": 0, "lo": 0, "hi": 10**6},
    {"name": "uniform_n20000_seed0", "generator": "uniform", "n": 20000, "seed": 0, "lo": 0, "hi": 10**6,
     "prefix": PREFIX_SWEEPS},
]


def make_input(w):
    if w["generator"] == "uniform":
        return inputs.uniform(w["n"], w["lo"], w["hi"], w["seed"])
    return getattr(inputs, w["generator"])(w["n"], w["seed"])


def sha(arr) -> str:
    return hashlib.sha256(np.ascontiguousarray(arr).tobytes()).hexdigest()


def solve_record(w, threads):
    a = make_input(w)
    rec = dict(w)
    rec["a_sha256"] = sha(a)
    t0 = time.time()
    g = oracle.greedy_init(a)
    rec.update({"greedy_objective": int(oracle.objective(a, g)), "greedy_tau_sha256": sha(g.astype(np.int32))})
    oracle.set_evaluation(threads, True)
    try:
        if w.get("prefix"):
            p = oracle.dgs_parallel(a, init=oracle.INIT_USER, init_tau=g, max_sweeps=w["prefix"],
                                    trace_cap=w["prefix"])
            rec["prefix_result"] = {"sweeps": int(p.sweeps), "status": int(p.status), "objective": int(p.objective),
                                    "tau_sha256": sha(p.tau.astype(np.int32)),
                                    "trace_accepted": p.trace_accepted.tolist(),
                                    "trace_applied": p.trace_applied.tolist(),
                                    "trace_objective": p.trace_objective.tolist()}
            print(w["name"], "prefix", rec["prefix_result"]["objective"], round(time.time() - t0, 1), flush=True)
        # the greedy start computed above, passed in as the start (the same solve as init=INIT_GREEDY)
        r = oracle.dgs_parallel(a, init=oracle.INIT_USER, init_tau=g, trace_cap=PREFIX_SWEEPS)
    finally:
        oracle.set_evaluation(1, False)
    dt = time.time() - t0
    rec.update({"status": int(r.status), "objective": int(r.objective), "sweeps": int(r.sweeps),
                "swaps_applied": int(r.swaps_applied), "tau_sha256": sha(r.tau.astype(np.int32)),
                "trace_objective_first": r.trace_objective.tolist(),
                "oracle_seconds": round(dt, 1), "oracle_threads": threads})
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    names = args.names or [w["name"] for w in WORKLOADS]
    for name in names:
        w = next(x for x in WORKLOADS if x["name"] == name)
        rec = solve_record(w, args.threads)
        print(rec["name"], {k: rec[k] for k in ("objective", "sweeps", "swaps_applied", "oracle_seconds")},
              flush=True)
        out = {"workloads": []}
        if os.path.exists(PATH):
            with open(PATH) as f:
                out = json.load(f)
        out["_source"] = ("oracle.dgs_parallel (plain C, Algorithms 2-4 with readings R1-R5), greedy start; "
                          "written by tests/golden/make_bench_golden.py")
        out["workloads"] = [x for x in out["workloads"] if x["name"] != name] + [rec]
        order = [x["name"] for x in WORKLOADS]
        out["workloads"].sort(key=lambda x: order.index(x["name"]))
        with open(PATH + ".tmp", "w") as f:
            json.dump(out, f, indent=1)
        os.replace(PATH + ".tmp", PATH)


if __name__ == "__main__":
    main()
