"""Record the FP64 oracle's own pass counts to tolerance on the benchmark
workloads (grid-blob image-like OT instances), for scaling a bounded CPU
sample of passes to solves/s.  Calls only the oracle (and the seeded input
generators).  Writes oracle/reference_counts.json.

usage: python oracle/reference_counts.py grid64 1e-6
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2407_19689_gb300 import instances as I  # noqa: E402

OUT = os.path.join(ROOT, "oracle", "reference_counts.json")


def run(name: str, tol: float):
    G = int(name.replace("grid", ""))
    ins = I.grid_blob_instance(G, I.seed_for(1, 0))
    C32 = ins.C.astype(np.float32).astype(np.float64)   # the FP32 cost the GPU path reads
    t = time.time()
    r = oracle.solve(C32, ins.f, ins.g, oracle.Options(tol=tol))
    rec = {"passes": r.passes, "iters": r.iters, "restarts": r.restarts, "status": r.status,
           "primal_obj": r.primal_obj, "rel_kkt": r.rel_kkt, "seconds_single_thread": time.time() - t}
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    data.setdefault(name, {})[f"{tol:g}"] = rec
    with open(OUT, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    print(name, tol, rec)


if __name__ == "__main__":
    run(sys.argv[1], float(sys.argv[2]))
