"""Writes tests/golden/synth_T65536.json: the FP64 CPU oracle's solution of the synthetic
scaling workload at its full horizon (x+ = A x + B u + 0.1 tanh(W x), n = 32, m = 8,
matrices from seed 0, x0 = synth_x0(0), T = 65536, interior point with the multiplier form
of the co-states, default tolerances), stored as its report, the cost and every 4096th row
of x and u (the whole trajectory is 20 MB).  The solve takes hours on one core, so the GPU
result at this size is compared with these stored samples.

Calls only oracle/ and the workload generator:  python tests/golden/synth_reference.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2409_20027_gb300 import workloads as W  # noqa: E402

T = 65536
EVERY = 4096
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_T65536.json")


def main():
    t0 = time.time()
    r = O.solve_ip(W.synth(0), W.synth_x0(0), T, opts=O.Options(costate_mode=1))
    rows = list(range(0, T + 1, EVERY))
    out = {"source": "oracle/ptn_oracle.c via oracle.solve_ip (FP64, serial), this script",
           "workload": "synth(seed 0), x0 = synth_x0(0), T = 65536, IP, costate_mode 1, default options",
           "seconds": time.time() - t0, "info": r["info"], "rows": rows,
           "x": r["x"][rows].tolist(), "u": r["u"][[t for t in rows if t < T]].tolist()}
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(json.dumps(r["info"]))


if __name__ == "__main__":
    main()
