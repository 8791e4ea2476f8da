"""Runs decompositions and products with the op-counting build of the
library and writes the counters (one process per run: the build is chosen
when the library loads).

    GF2_COUNT_OPS=1 python tests/op_count_child.py jobs.npz out.json

jobs.npz holds, for job i, "kind_i" ("decompose" or "mmm"), the row-major
words "A_i" (and "B_i"), the sizes in "dims_i" (decompose: n, m; mmm: n, k,
m, flags, strassen cutoff).  Used by tests/test_gpu_op_counts.py.
"""
from __future__ import annotations

import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_1209_5198_gb300 as gf2  # noqa: E402


def main(jobs_path: str, out_path: str) -> None:
    assert gf2.COUNTING, "run with GF2_COUNT_OPS=1"
    jobs = np.load(jobs_path)
    out = []
    i = 0
    while f"kind_{i}" in jobs:
        kind = str(jobs[f"kind_{i}"])
        dims = [int(x) for x in jobs[f"dims_{i}"]]
        A = jobs[f"A_{i}"]
        gf2.op_counts(reset=True)
        if kind == "decompose":
            n, m = dims
            res = gf2.decompose(gf2.Mat.from_rowmajor(A, m))
            counts = gf2.op_counts(reset=True)
            r = int(res["rank"].item())
            out.append({"kind": kind, "counts": counts, "rank": r,
                        "pivcols": res["pivcols"][:r].cpu().numpy().tolist()})
        else:
            n, k, m, flags, cutoff = dims
            gf2.set_strassen_cutoff(cutoff)
            C = gf2.mmm(gf2.Mat.from_rowmajor(A, k), gf2.Mat.from_rowmajor(jobs[f"B_{i}"], m), flags=flags)
            counts = gf2.op_counts(reset=True)
            Cw = C.to_rowmajor()
            out.append({"kind": kind, "counts": counts, "C": [int(x) for x in Cw.reshape(-1)]})
        torch.cuda.synchronize()
        i += 1
    with open(out_path, "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
