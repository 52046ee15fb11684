"""Small drivers for kernel profiling (ncu) of the library's entry points.

    python -m paper_1106_5694_gb300.profile_kernels evaluate --n 10000 --workload peer
    python -m paper_1106_5694_gb300.profile_kernels solve    --n 10000 --workload peer

    python -m paper_1106_5694_gb300.profile_kernels batched  --count 1024 --lo 64 --hi 4096

`evaluate` computes the greedy start once, then calls dgs_evaluate `--repeat`
times on it (each call launches one full_evaluation_kernel); `solve` calls
dgs_solve_ex `--repeat` times; `batched` calls dgs_solve_batched `--repeat`
times on `--count` peer-shaped instances with n log-uniform in [lo, hi]
(leading blocks of four pool matrices, as bench.py builds them).  Inputs
come from the seeded generators.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None) -> int:
    import torch

    from paper_1106_5694_gb300 import binding as B
    from paper_1106_5694_gb300 import inputs

    p = argparse.ArgumentParser()
    p.add_argument("what", choices=["evaluate", "solve", "batched"])
    p.add_argument("--count", type=int, default=1024)
    p.add_argument("--lo", type=int, default=64)
    p.add_argument("--hi", type=int, default=4096)
    p.add_argument("--n", type=int, default=10000)
    p.add_argument("--workload", choices=["peer", "uniform"], default="peer")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--repeat", type=int, default=2)
    args = p.parse_args(argv)
    if args.what == "batched":
        import numpy as np

        ns = inputs.batched_sizes(args.count, args.lo, args.hi, seed=7)
        pool = [inputs.peer_shaped(args.hi, 500 + k) for k in range(4)]
        mats = [torch.from_numpy(np.ascontiguousarray(pool[k % 4][:n, :n])).cuda() for k, n in enumerate(ns)]
        for _ in range(args.repeat):
            st = B.dgs_solve_batched(mats)[0]
            assert st == B.DGS_OK, B.dgs_status_string(st)
        torch.cuda.synchronize()
        print(f"batched count={args.count} n in [{args.lo},{args.hi}]: ok")
        return 0
    a = inputs.peer_shaped(args.n, args.seed) if args.workload == "peer" else \
        inputs.uniform(args.n, 0, 10**6, args.seed)
    at = torch.from_numpy(a).cuda()
    if args.what == "evaluate":
        st, g = B.dgs_greedy_init(at)
        assert st == B.DGS_OK, B.dgs_status_string(st)
        for _ in range(args.repeat):
            st = B.dgs_evaluate(at, g)[0]
            assert st == B.DGS_OK, B.dgs_status_string(st)
    else:
        for _ in range(args.repeat):
            st = B.dgs_solve_ex(at)[0]
            assert st == B.DGS_OK, B.dgs_status_string(st)
    torch.cuda.synchronize()
    print(f"{args.what} n={args.n} {args.workload}: ok")
    return 0


if __name__ == "__main__":
    sys.exit(main())
