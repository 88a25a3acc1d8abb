"""Record how many squares the CPU FP64 oracle needs on the benchmark workloads --
TEST INFRASTRUCTURE ONLY.

The benchmark's CPU-baseline leg times a bounded sample of oracle iterations and
extrapolates to a full run; the number of squares of that full run is stored here,
computed by the oracle itself (one complete run per workload).  Run:
    python -m oracle.record_iteration_counts [N ...]
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

from oracle import sp2_oracle as o  # noqa: E402
from paper_1507_02087_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "iteration_counts.json")


def record(N: int, gap: float) -> dict:
    nocc = N // 2
    case = inputs.dense_gapped(N, nocc, gap=gap, seed=0, want_exact=False)
    t = time.perf_counter()
    res = o.sp2(case.F.numpy(), nocc)
    dt = time.perf_counter() - t
    # squares computed: one per recorded v (v_0 .. v_{n}) unless the guard ended the run
    squares = len(res.v)
    return {"N": N, "nocc": nocc, "gap": gap, "seed": 0, "n": res.n, "stop_reason": res.stop_reason,
            "squares": squares, "oracle_seconds": dt, "cores": os.cpu_count()}


def main(argv):
    sizes = [int(a) for a in argv] or [400, 8192]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for N in sizes:
        gap = 0.1 if N == 400 else 0.01
        key = f"dense_N{N}_nocc{N // 2}_gap{gap:g}_seed0"
        data[key] = record(N, gap)
        print(key, data[key], flush=True)
        json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
