"""numpy wrappers around the C oracle (test infrastructure only).

Every wrapper converts its arguments to contiguous numpy arrays of the
C function's types and calls it; no arithmetic of the method happens here
apart from the bookkeeping that assembles log T~ = log u + log K~ + log v
for the objective, which is the definition of T~ = diag(u) K~ diag(v)
(section 3.2, output line of Alg. 3 / Alg. 4).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sparsink_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libsparsink_oracle.so")
_lock = threading.Lock()
_lib = None

STOP_RESIDUAL = 0
STOP_DELTA_UV = 1


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain C, FP64, no contraction)."""
    src_mtime = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "sparsink_oracle.h")))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= src_mtime:
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class Problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("d", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p), ("C", C.c_void_p),
                ("cost_norm", C.c_int32), ("cost_scale", C.c_double), ("a", C.c_void_p), ("b", C.c_void_p),
                ("eps", C.c_double), ("lam", C.c_double), ("s", C.c_double),
                ("seed", C.c_uint64), ("pid", C.c_uint32), ("cost_kind", C.c_int32), ("eta", C.c_double),
                ("probs", C.c_int32)]


class Scalars(C.Structure):
    _fields_ = [("dmax64", C.c_double), ("dmax32", C.c_float), ("sum1", C.c_double),
                ("sum2", C.c_double), ("scale32", C.c_float), ("s32", C.c_float),
                ("gamma32", C.c_float), ("kappa32", C.c_float), ("inv2eta32", C.c_float), ("g2_32", C.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("residual", C.c_double),
                ("unreach_a", C.c_double), ("unreach_b", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build_oracle())
            P = C.c_void_p
            i32, i64, u32, u64, f64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
            _lib.orc_philox4x32_10.argtypes = [P, P, P]
            _lib.orc_draw24.argtypes = [u64, u32, u32, u32]
            _lib.orc_draw24.restype = u32
            _lib.orc_exp32_vec.argtypes = [P, P, i64]
            _lib.orc_cos32_vec.argtypes = [P, P, i64]
            _lib.orc_log32_vec.argtypes = [P, P, i64]
            _lib.orc_exact_sum_f32.argtypes = [P, i64]
            _lib.orc_exact_sum_f32.restype = f64
            _lib.orc_factors.argtypes = [P, P, P, P]
            _lib.orc_factors.restype = C.c_int
            _lib.orc_pstar_raw.argtypes = [P, P, P, P, i32, i32]
            _lib.orc_pstar_raw.restype = C.c_float
            _lib.orc_count.argtypes = [P, P, P, P, P]
            _lib.orc_count.restype = i64
            _lib.orc_sample_row.argtypes = [P, P, P, P, i32, P, P, P, P, P]
            _lib.orc_sample_row.restype = i32
            _lib.orc_sparsify.argtypes = [P] + [P] * 10 + [P]
            _lib.orc_sparsify.restype = i64
            _lib.orc_sparsify_skip.argtypes = [P] + [P] * 10 + [P]
            _lib.orc_sparsify_skip.restype = i64
            _lib.orc_log1m32_vec.argtypes = [P, P, i64]
            _lib.orc_skip_words.argtypes = [u64, u32, u32, u32, P]
            _lib.orc_colf_max.argtypes = [P, i32]
            _lib.orc_colf_max.restype = C.c_float
            _lib.orc_skip_row.argtypes = [P, P, P, P, C.c_float, i32, P, P, P, P, P]
            _lib.orc_skip_row.restype = i32
            _lib.orc_skip_count.argtypes = [P, P, P, P, P]
            _lib.orc_skip_count.restype = i64
            _lib.orc_dense_kernel.argtypes = [P, P, P]
            _lib.orc_dense_kernel.restype = C.c_int
            _lib.orc_sinkhorn_sparse.argtypes = [i32, i32, P, P, P, P, P, P, P, P, f64, f64, f64,
                                                 i32, i32, P, P, P, P, P]
            _lib.orc_sinkhorn_dense.argtypes = [i32, i32, P, P, P, f64, f64, f64, i32, i32, P, P,
                                                P, P, P]
            _lib.orc_sinkhorn_log_sparse.argtypes = [i32, i32, P, P, P, P, P, P, P, P, f64, f64,
                                                     f64, i32, i32, P, P, P, P, P]
            _lib.orc_objective_terms.argtypes = [i32, i32, P, P, P, P, P, P, P, P]
        return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# RNG and binary32 spec arithmetic
# --------------------------------------------------------------------------

def philox4x32_10(ctr, key):
    """Philox4x32-10 of each counter row ctr[k, 0:4] under key[0:2]."""
    lib = load()
    ctr = _c(np.atleast_2d(ctr), np.uint32)
    key = _c(key, np.uint32)
    out = np.empty_like(ctr)
    for k in range(ctr.shape[0]):
        lib.orc_philox4x32_10(_ptr(ctr[k]), _ptr(key), _ptr(out[k]))
    return out


def draw24(seed, pid, i, j):
    lib = load()
    i = np.atleast_1d(np.asarray(i, dtype=np.int64))
    j = np.atleast_1d(np.asarray(j, dtype=np.int64))
    i, j = np.broadcast_arrays(i, j)
    return np.array([lib.orc_draw24(seed, pid, int(a), int(b)) for a, b in zip(i.ravel(), j.ravel())],
                    dtype=np.uint32).reshape(i.shape)


def exp32(x):
    lib = load()
    x = _c(x, np.float32)
    y = np.empty_like(x)
    lib.orc_exp32_vec(_ptr(x), _ptr(y), x.size)
    return y


def log32(x):
    lib = load()
    x = _c(x, np.float32)
    y = np.empty_like(x)
    lib.orc_log32_vec(_ptr(x), _ptr(y), x.size)
    return y


def cos32(z):
    """Spec cos in binary32 on [0, pi/2] (the WFR decision path)."""
    lib = load()
    z = _c(np.ravel(z), np.float32)
    y = np.empty_like(z)
    lib.orc_cos32_vec(_ptr(z), _ptr(y), z.size)
    return y


def log1m32(q):
    """Spec log(1 - q) in binary32, 0 < q < 1 (skip sampler gaps)."""
    lib = load()
    q = _c(np.ravel(q), np.float32)
    y = np.empty_like(q)
    lib.orc_log1m32_vec(_ptr(q), _ptr(y), q.size)
    return y


def skip_words(seed, pid, i, t):
    """The two Philox words of candidate t of row i in the skip sampler."""
    lib = load()
    w = np.empty(2, np.uint32)
    lib.orc_skip_words(int(seed), int(pid), int(i), int(t), _ptr(w))
    return int(w[0]), int(w[1])


def exact_sum_f32(x):
    lib = load()
    x = _c(np.ravel(x), np.float32)
    return lib.orc_exact_sum_f32(_ptr(x), x.size)


# --------------------------------------------------------------------------
# Problems and sampling
# --------------------------------------------------------------------------

class OracleProblem:
    """Holds the numpy arrays of one problem alive for the C struct."""

    def __init__(self, a, b, eps, s, lam=math.inf, x=None, y=None, C_=None, cost_norm=1,
                 seed=0x5EED, pid=0, cost_scale=1.0, cost_kind="sqeuclid", eta=0.0, probs="paper"):
        """cost_kind: "sqeuclid" (squared Euclidean, or the matrix C_) or "wfr"
        (Wasserstein-Fisher-Rao with parameter eta; raw cost, cost_norm = 0).
        probs: "paper" (Eq. (pij-ot) / (pij-uot)) or "uniform" (p_ij = 1/(n m), the
        Rand-Sink control)."""
        self.a = _c(a, np.float64)
        self.b = _c(b, np.float64)
        self.x = _c(x, np.float64)
        self.y = _c(y, np.float64)
        self.C = _c(C_, np.float64)
        self.n, self.m = self.a.size, self.b.size
        self.d = 0 if self.x is None else (self.x.shape[1] if self.x.ndim == 2 else 1)
        self.eps, self.lam, self.s = float(eps), float(lam), float(s)
        self.cost_norm = int(cost_norm)
        self.cost_scale = float(cost_scale)
        self.seed, self.pid = int(seed), int(pid)
        self.cost_kind, self.eta = (1 if cost_kind == "wfr" else 0), float(eta)
        self.probs = {"paper": 0, "uniform": 1}[probs]
        self.struct = Problem(self.n, self.m, self.d, _ptr(self.x), _ptr(self.y), _ptr(self.C),
                              self.cost_norm, self.cost_scale, _ptr(self.a), _ptr(self.b), self.eps,
                              self.lam, self.s, self.seed, self.pid, self.cost_kind, self.eta, self.probs)
        self._factors = None

    @property
    def is_ot(self):
        return math.isinf(self.lam)

    def factors(self):
        if self._factors is None:
            lib = load()
            rowf = np.empty(self.n, np.float32)
            colf = np.empty(self.m, np.float32)
            S = Scalars()
            rc = lib.orc_factors(C.byref(self.struct), _ptr(rowf), _ptr(colf), C.byref(S))
            if rc != 0:
                raise ValueError(f"orc_factors failed ({rc})")
            self._factors = (rowf, colf, S)
        return self._factors

    def pstar_raw(self, i, j):
        lib = load()
        rowf, colf, S = self.factors()
        return lib.orc_pstar_raw(C.byref(self.struct), _ptr(rowf), _ptr(colf), C.byref(S), int(i), int(j))

    def count(self):
        lib = load()
        rowf, colf, S = self.factors()
        cnt = np.empty(self.n, np.int32)
        nnz = lib.orc_count(C.byref(self.struct), _ptr(rowf), _ptr(colf), C.byref(S), _ptr(cnt))
        return cnt, int(nnz)

    def sample_row(self, i):
        lib = load()
        rowf, colf, S = self.factors()
        m = self.m
        cols = np.empty(m, np.int32)
        val = np.empty(m, np.float64)
        logv = np.empty(m, np.float64)
        ps = np.empty(m, np.float32)
        cost = np.empty(m, np.float64)
        c = lib.orc_sample_row(C.byref(self.struct), _ptr(rowf), _ptr(colf), C.byref(S), int(i),
                               _ptr(cols), _ptr(val), _ptr(logv), _ptr(ps), _ptr(cost))
        return {"cols": cols[:c].copy(), "val": val[:c].copy(), "logval": logv[:c].copy(),
                "pstar": ps[:c].copy(), "cost": cost[:c].copy()}

    def skip_row(self, i):
        """Row i of the skip sampler's sketch."""
        lib = load()
        rowf, colf, S = self.factors()
        cmax = lib.orc_colf_max(_ptr(colf), self.m)
        m = self.m
        cols = np.empty(m, np.int32)
        val = np.empty(m, np.float64)
        logv = np.empty(m, np.float64)
        ps = np.empty(m, np.float32)
        cost = np.empty(m, np.float64)
        c = lib.orc_skip_row(C.byref(self.struct), _ptr(rowf), _ptr(colf), C.byref(S), cmax, int(i),
                             _ptr(cols), _ptr(val), _ptr(logv), _ptr(ps), _ptr(cost))
        return {"cols": cols[:c].copy(), "val": val[:c].copy(), "logval": logv[:c].copy(),
                "pstar": ps[:c].copy(), "cost": cost[:c].copy()}

    def skip_count(self):
        """Row counts of the skip sampler's sketch (O(sampled) work)."""
        lib = load()
        rowf, colf, S = self.factors()
        cnt = np.empty(self.n, np.int32)
        nnz = lib.orc_skip_count(C.byref(self.struct), _ptr(rowf), _ptr(colf), C.byref(S), _ptr(cnt))
        return cnt, int(nnz)

    def sparsify(self, sampler="element"):
        """Full sketch.  sampler: "element" (one decision per element) or
        "skip" (geometric skips with thinning)."""
        lib = load()
        if sampler == "skip":
            _, nnz = self.skip_count()
        else:
            _, nnz = self.count()
        n, m = self.n, self.m
        out = {
            "row_ptr": np.empty(n + 1, np.int32), "col_idx": np.empty(nnz, np.int32),
            "val": np.empty(nnz, np.float64), "logval": np.empty(nnz, np.float64),
            "pstar": np.empty(nnz, np.float32), "cost": np.empty(nnz, np.float64),
            "col_ptr": np.empty(m + 1, np.int32), "row_idx": np.empty(nnz, np.int32),
            "valT": np.empty(nnz, np.float64), "perm": np.empty(nnz, np.int32),
        }
        S = Scalars()
        k = ["row_ptr", "col_idx", "val", "logval", "pstar", "cost", "col_ptr", "row_idx", "valT", "perm"]
        fn = lib.orc_sparsify_skip if sampler == "skip" else lib.orc_sparsify
        got = fn(C.byref(self.struct), *[_ptr(out[x]) for x in k], C.byref(S))
        if got != nnz:
            raise RuntimeError("sparsify count mismatch")
        out["nnz"] = nnz
        out["logvalT"] = out["logval"][out["perm"]]
        out["scalars"] = S.as_dict()
        out["n"], out["m"] = n, m
        return out

    def dense_kernel(self):
        lib = load()
        K = np.empty((self.n, self.m), np.float64)
        Cn = np.empty((self.n, self.m), np.float64)
        if lib.orc_dense_kernel(C.byref(self.struct), _ptr(K), _ptr(Cn)) != 0:
            raise ValueError("bad problem")
        return K, Cn


# --------------------------------------------------------------------------
# Iterations and objective
# --------------------------------------------------------------------------

def sinkhorn_sparse(sk, a, b, eps, lam=math.inf, tol=1e-6, max_iter=1000, stop_rule=STOP_RESIDUAL,
                    u0=None, v0=None):
    lib = load()
    n, m = sk["n"], sk["m"]
    a, b = _c(a, np.float64), _c(b, np.float64)
    u0, v0 = _c(u0, np.float64), _c(v0, np.float64)
    u, v = np.empty(n), np.empty(m)
    info = SolveInfo()
    lib.orc_sinkhorn_sparse(n, m, _ptr(sk["row_ptr"]), _ptr(sk["col_idx"]), _ptr(sk["val"]),
                            _ptr(sk["col_ptr"]), _ptr(sk["row_idx"]), _ptr(sk["valT"]), _ptr(a),
                            _ptr(b), eps, lam, tol, max_iter, stop_rule, _ptr(u0), _ptr(v0), _ptr(u),
                            _ptr(v), C.byref(info))
    return u, v, info.as_dict()


def sinkhorn_dense(K, a, b, eps, lam=math.inf, tol=1e-6, max_iter=1000, stop_rule=STOP_RESIDUAL,
                   u0=None, v0=None):
    lib = load()
    K = _c(K, np.float64)
    n, m = K.shape
    a, b = _c(a, np.float64), _c(b, np.float64)
    u0, v0 = _c(u0, np.float64), _c(v0, np.float64)
    u, v = np.empty(n), np.empty(m)
    info = SolveInfo()
    lib.orc_sinkhorn_dense(n, m, _ptr(K), _ptr(a), _ptr(b), eps, lam, tol, max_iter, stop_rule,
                           _ptr(u0), _ptr(v0), _ptr(u), _ptr(v), C.byref(info))
    return u, v, info.as_dict()


def sinkhorn_log_sparse(sk, a, b, eps, lam=math.inf, tol=1e-6, max_iter=1000,
                        stop_rule=STOP_RESIDUAL, alpha0=None, beta0=None):
    lib = load()
    n, m = sk["n"], sk["m"]
    a, b = _c(a, np.float64), _c(b, np.float64)
    al0, be0 = _c(alpha0, np.float64), _c(beta0, np.float64)
    al, be = np.empty(n), np.empty(m)
    info = SolveInfo()
    lib.orc_sinkhorn_log_sparse(n, m, _ptr(sk["row_ptr"]), _ptr(sk["col_idx"]), _ptr(sk["logval"]),
                                _ptr(sk["col_ptr"]), _ptr(sk["row_idx"]), _ptr(sk["logvalT"]),
                                _ptr(a), _ptr(b), eps, lam, tol, max_iter, stop_rule, _ptr(al0),
                                _ptr(be0), _ptr(al), _ptr(be), C.byref(info))
    return al, be, info.as_dict()


def objective_terms(row_ptr, col_idx, logT, cost, pstar, a, b):
    """Returns dict(transport, neg_entropy, logp, mass, kl_a, kl_b)."""
    lib = load()
    row_ptr, col_idx = _c(row_ptr, np.int32), _c(col_idx, np.int32)
    logT, cost, pstar = _c(logT, np.float64), _c(cost, np.float64), _c(pstar, np.float32)
    a, b = _c(a, np.float64), _c(b, np.float64)
    out = np.zeros(7)
    lib.orc_objective_terms(a.size, b.size, _ptr(row_ptr), _ptr(col_idx), _ptr(logT), _ptr(cost),
                            _ptr(pstar), _ptr(a), _ptr(b), _ptr(out))
    return dict(zip(["transport", "neg_entropy", "logp", "mass", "kl_a", "kl_b"], out[:6].tolist()))


def _objective(terms, eps, lam):
    """R1 = <T,C> - eps H(T) (+ lam KL terms): the output line of Alg. 3/4.
    R2 adds eps sum T log p* (the sparse problem's own value, cost C~)."""
    r1 = terms["transport"] + eps * terms["neg_entropy"]
    if not math.isinf(lam):
        r1 += lam * (terms["kl_a"] + terms["kl_b"])
    return r1, r1 + eps * terms["logp"]


def _log_or_neginf(x):
    with np.errstate(divide="ignore"):
        return np.log(x)


def spar_sink(prob: OracleProblem, tol=1e-6, max_iter=1000, log_domain=False, stop_rule=STOP_RESIDUAL,
              sketch=None):
    """Alg. 3 (OT, lam = inf) or Alg. 4 (UOT): sketch, iterate, objective."""
    sk = prob.sparsify() if sketch is None else sketch
    a, b = prob.a, prob.b
    rows = np.repeat(np.arange(prob.n), np.diff(sk["row_ptr"]))
    if log_domain:
        al, be, info = sinkhorn_log_sparse(sk, a, b, prob.eps, prob.lam, tol, max_iter, stop_rule)
        logT = (al[rows] + be[sk["col_idx"]]) / prob.eps + sk["logval"]
        logu, logv = al / prob.eps, be / prob.eps
    else:
        u, v, info = sinkhorn_sparse(sk, a, b, prob.eps, prob.lam, tol, max_iter, stop_rule)
        logu, logv = _log_or_neginf(u), _log_or_neginf(v)
        logT = logu[rows] + _log_or_neginf(sk["val"]) + logv[sk["col_idx"]]   # K~ = 0 where WFR blocks
    terms = objective_terms(sk["row_ptr"], sk["col_idx"], logT, sk["cost"], sk["pstar"], a, b)
    r1, r2 = _objective(terms, prob.eps, prob.lam)
    return {"sketch": sk, "alpha": prob.eps * logu, "beta": prob.eps * logv, "info": info,
            "terms": terms, "obj": r1, "obj_sparse": r2}


def dense_sinkhorn(prob: OracleProblem, tol=1e-6, max_iter=1000, stop_rule=STOP_RESIDUAL, log_domain=False):
    """Alg. 1 / Alg. 2 on the dense kernel, with the same objective terms.
    log_domain=True runs the log-sum-exp iterations over the full support
    (log K = -C/eps), for the small eps at which K underflows."""
    K, Cn = prob.dense_kernel()
    n, m = K.shape
    row_ptr = (np.arange(n + 1) * m).astype(np.int32)
    col_idx = np.tile(np.arange(m, dtype=np.int32), n)
    if log_domain:
        lk = -Cn / prob.eps
        full = {"n": n, "m": m, "row_ptr": row_ptr, "col_idx": col_idx, "logval": lk.ravel(),
                "col_ptr": (np.arange(m + 1) * n).astype(np.int32),
                "row_idx": np.tile(np.arange(n, dtype=np.int32), m), "logvalT": lk.T.ravel()}
        al, be, info = sinkhorn_log_sparse(full, prob.a, prob.b, prob.eps, prob.lam, tol, max_iter, stop_rule)
        logT = ((al[:, None] + be[None, :]) / prob.eps + lk).ravel()
        terms = objective_terms(row_ptr, col_idx, logT, Cn.ravel(), np.ones(n * m, np.float32), prob.a, prob.b)
        r1, _ = _objective(terms, prob.eps, prob.lam)
        return {"alpha": al, "beta": be, "info": info, "terms": terms, "obj": r1, "K": K, "C": Cn}
    u, v, info = sinkhorn_dense(K, prob.a, prob.b, prob.eps, prob.lam, tol, max_iter, stop_rule)
    logu, logv = _log_or_neginf(u), _log_or_neginf(v)
    with np.errstate(divide="ignore"):
        logT = (logu[:, None] + np.log(K) + logv[None, :]).ravel()
    terms = objective_terms(row_ptr, col_idx, logT, Cn.ravel(), np.ones(n * m, np.float32),
                            prob.a, prob.b)
    r1, _ = _objective(terms, prob.eps, prob.lam)
    return {"alpha": prob.eps * logu, "beta": prob.eps * logv, "u": u, "v": v, "info": info,
            "terms": terms, "obj": r1, "K": K, "C": Cn}


__all__ = ["build_oracle", "load", "philox4x32_10", "draw24", "exp32", "log32", "log1m32", "skip_words", "cos32",
           "exact_sum_f32",
           "OracleProblem", "sinkhorn_sparse", "sinkhorn_dense", "sinkhorn_log_sparse",
           "objective_terms", "spar_sink", "dense_sinkhorn", "STOP_RESIDUAL", "STOP_DELTA_UV"]
