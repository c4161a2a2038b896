"""Writes ot_n200000_oracle.json: the FP64 oracle's Spar-Sink OT solve (log
domain, Alg. 3 with Alg. 1 in LSE form) of the 200000-point, 8-component
Gaussian-mixture workload in R^3 (eps = 0.01, s = 16 n ln n, tol 1e-5).

Calls only the oracle.  The inputs are the seeded generator's points and
weights rounded to binary32, exactly as the GPU receives them.  Takes about
15 minutes on 8 cores.  Usage: python tests/golden/make_ot_n200000_oracle.py
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_2306_06581_gb300 import inputs  # noqa: E402


def main():
    w = inputs.ot_n200000()
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    P = orc.OracleProblem(f(w.a), f(w.b), w.eps, w.s, math.inf, x=f(w.x), y=f(w.y), seed=w.seed, pid=w.pid)
    t0 = time.time()
    sk = P.sparsify()
    t1 = time.time()
    o = orc.spar_sink(P, tol=w.tol, max_iter=20000, log_domain=True, sketch=sk)
    t2 = time.time()
    rows = [0, 1, 777, 54321, 99999, 123456, 199999]
    out = {
        "workload": w.name, "n": w.n, "m": w.m, "d": w.d, "eps": w.eps, "s": w.s, "tol": w.tol,
        "seed": w.seed, "pid": w.pid, "nnz": int(sk["nnz"]),
        "row_nnz": {str(i): int(sk["row_ptr"][i + 1] - sk["row_ptr"][i]) for i in rows},
        "iters": int(o["info"]["iters"]), "status": int(o["info"]["status"]),
        "residual": float(o["info"]["residual"]), "unreach_a": float(o["info"]["unreach_a"]),
        "unreach_b": float(o["info"]["unreach_b"]),
        "terms": {k: float(v) for k, v in o["terms"].items()},
        "obj": float(o["obj"]), "obj_sparse": float(o["obj_sparse"]),
        "seconds": {"sketch": t1 - t0, "solve": t2 - t1},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ot_n200000_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
