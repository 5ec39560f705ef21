"""Writes oracle_ranks.json: the TT ranks the FP64 oracle's TT-SVD finds for each
workload's coefficient tensor (tol 1e-10), the norm ||C||_F, and per-theta accuracy of
the oracle's own K~ against dense K on a 300 x 300 subsample (the interpolation floor).

Calls only oracle/ and the seeded input generators. C3 needs ~6 minutes and ~20 GB RAM.
Usage: python tests/golden/make_oracle_ranks.py [c1 c2 c3]
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle.pttk_oracle as o  # noqa: E402
from paper_2406_06344_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_ranks.json")


def main(names):
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for name in names:
        w = W.WORKLOADS[name]
        cores, ranks, C = o.build_offline(w.kernel, w.d, w.dtheta, w.mode_boxes(), w.n, w.tol)
        X, Y = W.sources(w, 300), W.targets(w, 300)
        errs = []
        for th in W.thetas(w, 4):
            U, M, V = o.instantiate(cores, w.d, w.dtheta, w.mode_boxes(), th, X, Y)
            errs.append(o.rel_fro(o.kernel_matrix(w.kernel, X, Y, th), U @ M @ V.T))
        data[name] = {"ranks": ranks, "norm_C": float(np.linalg.norm(C.ravel())), "tol": w.tol,
                      "rel_err_vs_dense_first4_theta": errs}
        print(name, data[name], flush=True)
        json.dump(data, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c1", "c2", "c3"])
