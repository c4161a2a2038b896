"""ibp_oracle.py -- plain FP64 reference of IBP and Spar-IBP (fixed-support
Wasserstein barycenters, the paper's appendix on barycenters).

TEST INFRASTRUCTURE ONLY: used by the tests; shares no code with the CUDA
library.

- IBP (the appendix's IBP algorithm, after Benamou et al. 2015): from q^0 = 1/n and u_k^0 = 1,
  every iteration updates, for each measure k, v_k = b_k / (K_k^T u_k), then
  q = prod_k (K_k v_k)^{w_k}, then u_k = q / (K_k v_k) with the new q; it
  stops when ||q^t - q^{t-1}||_1 <= tol.  (As printed, the listing forms u_k
  from the previous q before q is updated; taken literally that order leaves
  a common scale of the u_k oscillating with period 6 -- with one measure
  c_t = c_{t-1} / c_{t-2} -- and never converges, so the cited algorithm's
  order is used.  Both orders have the same fixed points.)
- Spar-IBP (the appendix's Spar-IBP algorithm): every K_k is replaced by its
  sketch of Eq. (pois) with p_{k,ij} = sqrt(b_{k,j}) / (n sum_j sqrt(b_{k,j})),
  which is the balanced-OT probability of Eq. (pij-ot) with a uniform source
  weight a = 1/n; the sketches are drawn by the oracle's sampler with problem
  id k.
- Readings where the algorithm is silent: a zero (K_k v_k)_i (an empty row
  of a sketch) gives q_i = 0 and u_{k,i} = 0; a zero (K_k^T u_k)_j gives
  v_{k,j} = 0 (that column's mass cannot be moved, as in the Spar-Sink
  iterations).
Pinned by tests/test_oracle_ibp.py.
"""
import math

import numpy as np
import scipy.sparse as sp

from .oracle import OracleProblem


def _safe_div(num, den):
    out = np.zeros_like(num, dtype=np.float64)
    ok = den > 0
    out[ok] = num[ok] / den[ok]
    return out


def ibp(Ks, bs, w, tol=1e-9, max_iter=10000):
    """IBP on kernels Ks (dense arrays or scipy sparse, each n x n_k), target
    measures bs and weights w.  Returns (q, info) with info = {iters, delta,
    u, v}."""
    m = len(Ks)
    n = Ks[0].shape[0]
    w = np.asarray(w, np.float64)
    q = np.full(n, 1.0 / n)
    us = [np.ones(n) for _ in range(m)]
    vs = [None] * m
    delta = math.inf
    t = 0
    while t < max_iter:
        t += 1
        Kv = []
        for k in range(m):
            vs[k] = _safe_div(np.asarray(bs[k], np.float64), Ks[k].T @ us[k])
            Kv.append(np.asarray(Ks[k] @ vs[k], np.float64))
        logq = np.zeros(n)
        zero = np.zeros(n, bool)
        for k in range(m):
            zero |= Kv[k] <= 0
            logq += w[k] * np.log(np.where(Kv[k] > 0, Kv[k], 1.0))
        qn = np.where(zero, 0.0, np.exp(logq))
        for k in range(m):
            us[k] = _safe_div(qn, Kv[k])
        delta = float(np.abs(qn - q).sum())
        q = qn
        if delta <= tol:
            break
    return q, {"iters": t, "delta": delta, "u": us, "v": vs}


def spar_ibp_sketches(x, bs, eps, s, seed=0x5EED, cost_norm=1):
    """The sketches K~_k of Spar-IBP on the shared support x (n x d), as scipy
    CSR matrices, and the oracle sketches themselves."""
    n = x.shape[0]
    a = np.full(n, 1.0 / n)
    mats, sks = [], []
    for k, b in enumerate(bs):
        P = OracleProblem(a, b, eps, s, math.inf, x=x, y=x, seed=seed, pid=k, cost_norm=cost_norm)
        sk = P.sparsify()
        mats.append(sp.csr_matrix((sk["val"], sk["col_idx"], sk["row_ptr"]), shape=(n, len(b))))
        sks.append(sk)
    return mats, sks


def dense_kernels(x, bs, eps, cost_norm=1):
    """K_k = exp(-C / eps) with the oracle's normalised cost (shared support)."""
    n = x.shape[0]
    a = np.full(n, 1.0 / n)
    out = []
    for b in bs:
        K, _ = OracleProblem(a, b, eps, 1.0, math.inf, x=x, y=x, cost_norm=cost_norm).dense_kernel()
        out.append(K)
    return out


def spar_ibp(x, bs, w, eps, s, tol=1e-9, max_iter=10000, seed=0x5EED):
    """Spar-IBP: IBP on the sketches.  Returns (q, info)."""
    mats, _ = spar_ibp_sketches(x, bs, eps, s, seed)
    return ibp(mats, bs, w, tol, max_iter)
