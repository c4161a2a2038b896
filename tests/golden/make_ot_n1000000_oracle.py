"""Writes ot_n1000000_oracle.json: the FP64 oracle's Spar-Sink OT solve (log
domain, Alg. 3 with Alg. 1 in LSE form) of the 1,000,000-point,
16-component Gaussian-mixture workload in R^3 (eps = 0.01, s = 16 n ln n,
tol 1e-5), sketched with the skip sampler (geometric gaps with thinning) and
the workload's cost divided by its maximum over all n*m pairs.

Calls only the oracle.  The inputs are the seeded generator's points and
weights rounded to binary32, exactly as the GPU receives them.  Besides the
objective terms it stores, for a fixed sample of rows and columns, the row
counts of the sketch and the potentials with the gauge of OT fixed by
sum_i a_i alpha_i = sum_j b_j beta_j (OT potentials are unique only up to
(alpha + c, beta - c)).  Takes about half an hour and 15 GB of memory on 8
cores.  Usage: python tests/golden/make_ot_n1000000_oracle.py
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

# fixed sample of rows / columns whose counts and potentials are stored
SAMPLE = [0, 1, 2, 777, 4096, 54321, 99999, 123456, 250000, 314159, 499999, 500000, 654321, 777777, 888888,
          999998, 999999]


def gauge_fixed(a, b, al, be):
    """(alpha + c, beta - c) with c chosen so that sum a alpha = sum b beta
    over the reachable entries."""
    fa, fb = np.isfinite(al), np.isfinite(be)
    c = (np.dot(b[fb], be[fb]) - np.dot(a[fa], al[fa])) / 2.0
    return al + c, be - c


def main():
    w = inputs.ot_n1000000()
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    a, b = f(w.a), f(w.b)
    P = orc.OracleProblem(a, b, w.eps, w.s, math.inf, x=f(w.x), y=f(w.y), seed=w.seed, pid=w.pid)
    t0 = time.time()
    sk = P.sparsify(sampler="skip")
    t1 = time.time()
    o = orc.spar_sink(P, tol=w.tol, max_iter=20000, log_domain=True, sketch=sk)
    t2 = time.time()
    al, be = gauge_fixed(a, b, o["alpha"], o["beta"])
    rp, cp = sk["row_ptr"], sk["col_ptr"]
    out = {
        "workload": w.name, "n": w.n, "m": w.m, "d": w.d, "eps": w.eps, "s": w.s, "tol": w.tol,
        "seed": w.seed, "pid": w.pid, "sampler": "skip", "nnz": int(sk["nnz"]),
        "cost_max32": float(sk["scalars"]["dmax32"]),
        "row_nnz": {str(i): int(rp[i + 1] - rp[i]) for i in SAMPLE},
        "col_nnz": {str(j): int(cp[j + 1] - cp[j]) for j in SAMPLE},
        "alpha": {str(i): float(al[i]) for i in SAMPLE},
        "beta": {str(j): float(be[j]) for j in SAMPLE},
        "iters": int(o["info"]["iters"]), "status": int(o["info"]["status"]),
        "residual": float(o["info"]["residual"]), "unreach_a": float(o["info"]["unreach_a"]),
        "unreach_b": float(o["info"]["unreach_b"]),
        "terms": {k: float(v) for k, v in o["terms"].items()},
        "obj": float(o["obj"]), "obj_sparse": float(o["obj_sparse"]),
        "seconds": {"sketch": t1 - t0, "solve": t2 - t1},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ot_n1000000_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k not in ("alpha", "beta")}))


if __name__ == "__main__":
    main()
