"""Python binding of libsparsink.so (include/sparsink.h).

Argument marshalling only: tensors are checked for dtype/contiguity, moved to
the GPU when given on the host, and their device pointers, sizes and the
current CUDA stream are passed to the C ABI.  Every step of the method runs in
the CUDA library; there is no CPU fallback -- without the built library these
functions raise.

Function names are those of the C ABI: ``sinkhorn_dense``, ``sparsify_kernel``,
``spar_sink_ot``, ``spar_sink_uot`` and ``sps_workspace_bytes``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from dataclasses import dataclass

import numpy as np

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsparsink.so")

SPS_OK, SPS_NOT_CONVERGED, SPS_ERR_INVALID_ARG, SPS_ERR_WORKSPACE, SPS_ERR_CAPACITY, SPS_ERR_NUMERIC, SPS_ERR_CUDA = range(7)
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", 2: "ERR_INVALID_ARG", 3: "ERR_WORKSPACE", 4: "ERR_CAPACITY",
                5: "ERR_NUMERIC", 6: "ERR_CUDA"}
F64, F32, BF16, F16 = 0, 1, 2, 3
DTYPE_CODES = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16}
COST_RAW, COST_MAXNORM, COST_SCALE = 0, 1, 2
COST_KINDS = {"sqeuclid": 0, "wfr": 1}
PROBS = {"paper": 0, "equal": 1}
STOP_RESIDUAL, STOP_DELTA_UV = 0, 1
OP_SPARSIFY, OP_SPAR_SINK, OP_DENSE = 0, 1, 2


class SpsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("d", C.c_int32), ("x", C.c_void_p), ("y", C.c_void_p),
                ("C", C.c_void_p), ("cost_norm", C.c_int32), ("cost_scale", C.c_double), ("a", C.c_void_p),
                ("b", C.c_void_p), ("dtype", C.c_int32), ("cost_kind", C.c_int32), ("eta", C.c_double)]


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("lam", C.c_double), ("s", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("check_every", C.c_int32), ("stop_rule", C.c_int32),
                ("seed", C.c_uint64), ("problem_id", C.c_uint32), ("kdtype", C.c_int32),
                ("log_domain", C.c_int32), ("absorb_tau", C.c_double), ("init_alpha", C.c_void_p),
                ("init_beta", C.c_void_p), ("gather_mode", C.c_int32), ("sketch_mode", C.c_int32),
                ("sampler", C.c_int32), ("probs", C.c_int32)]

GATHER_AUTO, GATHER_DIRECT, GATHER_STAGED = 0, 1, 2
PASS_DIRECT, PASS_STAGED, PASS_STAGED_FALLBACK = 0, 1, 2


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("residual", C.c_double), ("obj", C.c_double),
                ("obj_sparse", C.c_double), ("transport", C.c_double), ("neg_entropy", C.c_double),
                ("logp", C.c_double), ("mass", C.c_double), ("kl_a", C.c_double), ("kl_b", C.c_double),
                ("unreach_a", C.c_double), ("unreach_b", C.c_double), ("nnz", C.c_int64),
                ("n_absorb", C.c_int32), ("ms_sketch", C.c_float), ("ms_iter", C.c_float),
                ("ms_obj", C.c_float), ("launches", C.c_int32), ("iters_enqueued", C.c_int32),
                ("gather", C.c_int32), ("ms_setup", C.c_float), ("stream_bytes", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Sketch(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("nnz", C.c_int64), ("capacity", C.c_int64),
                ("kdtype", C.c_int32), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("col_ptr", C.c_void_p), ("row_idx", C.c_void_p), ("valT", C.c_void_p), ("csr_pos", C.c_void_p),
                ("sum1", C.c_double), ("sum2", C.c_double)]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2306_06581_gb300.build.build() "
                                   "(or __graft_entry__.build()); there is no CPU fallback")
            L = C.CDLL(LIB_PATH)
            P = C.c_void_p
            L.sps_workspace_bytes.argtypes = [P, P, C.c_int32]
            L.sps_workspace_bytes.restype = C.c_size_t
            for name in ("sinkhorn_dense", "spar_sink_ot", "spar_sink_uot"):
                f = getattr(L, name)
                f.argtypes = [P, P, P, C.c_size_t, P, P, P, P]
                f.restype = C.c_int
            L.sparsify_kernel.argtypes = [P, P, P, C.c_size_t, P, P]
            L.sparsify_kernel.restype = C.c_int
            L.sps_last_error.restype = C.c_char_p
            L.sps_version.restype = C.c_char_p
            _lib = L
        return _lib


def last_error() -> str:
    return lib().sps_last_error().decode()


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _dev(t, dtype, device):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    if t.dtype != dtype:
        t = t.to(dtype)
    if t.device != device:
        t = t.to(device, non_blocking=t.is_pinned())
    return t.contiguous()


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


@dataclass
class Marshalled:
    prob: Problem
    keep: tuple


def make_problem(a, b, x=None, y=None, C_=None, dtype="f32", cost_norm=COST_MAXNORM, cost_scale=1.0, device=None,
                 cost_kind="sqeuclid", eta=0.0):
    """Device copies of the inputs in `dtype` and the sps_problem struct.
    cost_kind "wfr" is the Wasserstein-Fisher-Rao cost with length scale eta
    (points, raw cost: cost_norm = COST_RAW)."""
    device = torch.device("cuda") if device is None else torch.device(device)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    a, b = _dev(a, tdt, device), _dev(b, tdt, device)
    x, y, C_ = _dev(x, tdt, device), _dev(y, tdt, device), _dev(C_, tdt, device)
    n, m = a.numel(), b.numel()
    d = 0 if x is None else (x.shape[1] if x.dim() == 2 else 1)
    p = Problem(n, m, d, _ptr(x), _ptr(y), _ptr(C_), cost_norm, float(cost_scale), _ptr(a), _ptr(b),
                F64 if dtype == "f64" else F32, COST_KINDS[cost_kind] if isinstance(cost_kind, str) else int(cost_kind),
                float(eta))
    return Marshalled(p, (a, b, x, y, C_))


SAMPLERS = {"element": 0, "skip": 1}


def make_params(eps, lam=math.inf, s=1.0, tol=1e-6, max_iter=1000, check_every=0, stop_rule=STOP_RESIDUAL,
                seed=0x5EED, problem_id=0, kdtype="f32", log_domain=0, absorb_tau=0.0, init_alpha=None,
                init_beta=None, gather_mode=GATHER_AUTO, sketch_mode=0, sampler="element", probs="paper"):
    return Params(float(eps), float(lam), float(s), float(tol), int(max_iter), int(check_every), int(stop_rule),
                  int(seed) & ((1 << 64) - 1), int(problem_id), DTYPE_CODES[kdtype] if isinstance(kdtype, str) else kdtype,
                  int(log_domain), float(absorb_tau), _ptr(init_alpha), _ptr(init_beta), int(gather_mode),
                  int(sketch_mode), SAMPLERS[sampler] if isinstance(sampler, str) else int(sampler),
                  PROBS[probs] if isinstance(probs, str) else int(probs))


def sps_workspace_bytes(prob: Problem, prm: Params, op: int) -> int:
    return int(lib().sps_workspace_bytes(C.byref(prob), C.byref(prm), op))


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _workspace(nbytes, device, workspace=None):
    if workspace is not None and workspace.numel() >= nbytes:
        return workspace
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def _check(status, allow_not_converged=True):
    if status == SPS_OK or (allow_not_converged and status == SPS_NOT_CONVERGED):
        return
    raise SpsError(status, last_error())


def _solve(fn_name, prob: Problem, prm: Params, device, op, workspace=None, raise_on_error=True):
    nbytes = sps_workspace_bytes(prob, prm, op)
    if nbytes == 0:
        raise SpsError(SPS_ERR_INVALID_ARG, last_error())
    ws = _workspace(nbytes, device, workspace)
    it_dtype = torch.float64 if prm.kdtype == F64 else torch.float32
    alpha = torch.empty(prob.n, dtype=it_dtype, device=device)
    beta = torch.empty(prob.m, dtype=it_dtype, device=device)
    res = Result()
    st = getattr(lib(), fn_name)(C.byref(prob), C.byref(prm), _ptr(ws), nbytes, _ptr(alpha), _ptr(beta),
                                 C.byref(res), _stream())
    if raise_on_error:
        _check(st)
    out = res.as_dict()
    out["status_code"] = st
    out["alpha"], out["beta"] = alpha, beta
    out["workspace"] = ws
    return out


# ---------------------------------------------------------------------------
# public calls (names of the C ABI)
# ---------------------------------------------------------------------------

def spar_sink_ot(a, b, x=None, y=None, C_=None, *, eps, s, tol=1e-6, max_iter=1000, dtype="f32", kdtype=None,
                 seed=0x5EED, problem_id=0, cost_norm=COST_MAXNORM, cost_scale=1.0, stop_rule=STOP_RESIDUAL,
                 check_every=0, init_alpha=None, init_beta=None, log_domain=0, absorb_tau=0.0, gather_mode=0, sketch_mode=0, workspace=None,
                 device=None, raise_on_error=True, sampler="element", cost_kind="sqeuclid", eta=0.0, probs="paper"):
    """Alg. 3: importance-sparsified Sinkhorn for balanced OT.  sampler="skip"
    draws the sketch by geometric gaps with thinning (work proportional to the
    sampled count; the same law as the per-element decisions).  probs="equal"
    samples every element with p_ij = 1/(n m) (the Rand-Sink control)."""
    M = make_problem(a, b, x, y, C_, dtype, cost_norm, cost_scale, device, cost_kind, eta)
    dev = M.keep[0].device
    kd = kdtype or dtype
    it = torch.float64 if kd == "f64" else torch.float32
    ia, ib = _dev(init_alpha, it, dev), _dev(init_beta, it, dev)
    prm = make_params(eps, math.inf, s, tol, max_iter, check_every, stop_rule, seed, problem_id, kd, log_domain,
                      absorb_tau, ia, ib, gather_mode, sketch_mode, sampler, probs)
    return _solve("spar_sink_ot", M.prob, prm, dev, OP_SPAR_SINK, workspace, raise_on_error)


def spar_sink_uot(a, b, x=None, y=None, C_=None, *, eps, lam, s, tol=1e-6, max_iter=1000, dtype="f32", kdtype=None,
                  seed=0x5EED, problem_id=0, cost_norm=COST_MAXNORM, cost_scale=1.0, stop_rule=STOP_RESIDUAL,
                  check_every=0, init_alpha=None, init_beta=None, log_domain=0, absorb_tau=0.0, gather_mode=0, sketch_mode=0, workspace=None,
                  device=None, raise_on_error=True, sampler="element", cost_kind="sqeuclid", eta=0.0, probs="paper"):
    """Alg. 4: importance-sparsified Sinkhorn for UOT with KL penalty lam.
    sampler="skip" draws the sketch by geometric gaps with thinning;
    cost_kind="wfr" uses the Wasserstein-Fisher-Rao cost (length scale eta,
    cost_norm=COST_RAW); probs="equal" samples with p_ij = 1/(n m)."""
    M = make_problem(a, b, x, y, C_, dtype, cost_norm, cost_scale, device, cost_kind, eta)
    dev = M.keep[0].device
    kd = kdtype or dtype
    it = torch.float64 if kd == "f64" else torch.float32
    ia, ib = _dev(init_alpha, it, dev), _dev(init_beta, it, dev)
    prm = make_params(eps, lam, s, tol, max_iter, check_every, stop_rule, seed, problem_id, kd, log_domain,
                      absorb_tau, ia, ib, gather_mode, sketch_mode, sampler, probs)
    return _solve("spar_sink_uot", M.prob, prm, dev, OP_SPAR_SINK, workspace, raise_on_error)


def sinkhorn_dense(a, b, x=None, y=None, C_=None, *, eps, lam=math.inf, tol=1e-6, max_iter=1000, dtype="f32",
                   cost_norm=COST_MAXNORM, cost_scale=1.0, stop_rule=STOP_RESIDUAL, check_every=0, log_domain=0,
                   init_alpha=None, init_beta=None, workspace=None, device=None, raise_on_error=True):
    """Alg. 1 (lam = inf) / Alg. 2 with K = exp(-C/eps) recomputed on the fly;
    log_domain=1 iterates the potentials in log-sum-exp form (binary32)."""
    M = make_problem(a, b, x, y, C_, dtype, cost_norm, cost_scale, device)
    dev = M.keep[0].device
    it = torch.float64 if dtype == "f64" else torch.float32
    ia, ib = _dev(init_alpha, it, dev), _dev(init_beta, it, dev)
    prm = make_params(eps, lam, 1.0, tol, max_iter, check_every, stop_rule, 0, 0, dtype, log_domain, 0.0, ia, ib)
    return _solve("sinkhorn_dense", M.prob, prm, dev, OP_DENSE, workspace, raise_on_error)


_NP_DT = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}


def sparsify_kernel(a, b, x=None, y=None, C_=None, *, eps, s, lam=math.inf, dtype="f32", kdtype=None, seed=0x5EED,
                    problem_id=0, cost_norm=COST_MAXNORM, cost_scale=1.0, sketch_mode=0, workspace=None,
                    device=None, sampler="element", cost_kind="sqeuclid", eta=0.0, probs="paper", log_domain=0):
    """Eq. (pois) sketch K~ as CSR + CSC tensor views (copied out of the workspace).
    log_domain only changes the params passed (the sketch is the same)."""
    M = make_problem(a, b, x, y, C_, dtype, cost_norm, cost_scale, device, cost_kind, eta)
    dev = M.keep[0].device
    kd = kdtype or dtype
    prm = make_params(eps, lam, s, 0.0, 1, 0, 0, seed, problem_id, kd, log_domain=log_domain, sketch_mode=sketch_mode,
                      sampler=sampler, probs=probs)
    nbytes = sps_workspace_bytes(M.prob, prm, OP_SPARSIFY)
    if nbytes == 0:
        raise SpsError(SPS_ERR_INVALID_ARG, last_error())
    ws = _workspace(nbytes, dev, workspace)
    sk = Sketch()
    st = lib().sparsify_kernel(C.byref(M.prob), C.byref(prm), _ptr(ws), nbytes, C.byref(sk), _stream())
    _check(st, allow_not_converged=False)
    base = ws.data_ptr()
    nnz = int(sk.nnz)
    vdt = _NP_DT[sk.kdtype]

    def view(ptr, count, dt):
        off = ptr - base
        esz = torch.empty((), dtype=dt).element_size()
        return ws[off:off + count * esz].view(dt).clone()

    n, m = M.prob.n, M.prob.m
    return {"nnz": nnz, "capacity": int(sk.capacity),
            "row_ptr": view(sk.row_ptr, n + 1, torch.int32), "col_idx": view(sk.col_idx, nnz, torch.int32),
            "val": view(sk.val, nnz, vdt), "col_ptr": view(sk.col_ptr, m + 1, torch.int32),
            "row_idx": view(sk.row_idx, nnz, torch.int32), "valT": view(sk.valT, nnz, vdt),
            "csr_pos": view(sk.csr_pos, nnz, torch.int32), "sum1": sk.sum1, "sum2": sk.sum2}


def spar_sink_ot_noalloc(a, b, x=None, y=None, C_=None, *, eps, s, tol=1e-6, max_iter=1000, dtype="f32",
                         kdtype=None, seed=0x5EED, problem_id=0, cost_norm=COST_MAXNORM, cost_scale=1.0,
                         stop_rule=STOP_RESIDUAL, check_every=0, device=None, raise_on_error=True):
    """Alg. 3 through the entry point that takes no workspace and allocates no
    device memory (its scratch is a fixed static array inside the library, so
    only problems that fit it are accepted).  Inputs are moved to the device
    here; callers that must not allocate pass device tensors."""
    M = make_problem(a, b, x, y, C_, dtype, cost_norm, cost_scale, device)
    dev = M.keep[0].device
    kd = kdtype or dtype
    prm = make_params(eps, math.inf, s, tol, max_iter, check_every, stop_rule, seed, problem_id, kd)
    it_dtype = torch.float64 if prm.kdtype == F64 else torch.float32
    alpha = torch.empty(M.prob.n, dtype=it_dtype, device=dev)
    beta = torch.empty(M.prob.m, dtype=it_dtype, device=dev)
    res = Result()
    f = lib().spar_sink_ot_noalloc
    f.argtypes = [C.c_void_p] * 6
    f.restype = C.c_int
    st = f(C.byref(M.prob), C.byref(prm), _ptr(alpha), _ptr(beta), C.byref(res), _stream())
    if raise_on_error:
        _check(st)
    out = res.as_dict()
    out["status_code"] = st
    out["alpha"], out["beta"] = alpha, beta
    return out


def version() -> str:
    return lib().sps_version().decode()


# ---------------------------------------------------------------------------
# Wasserstein barycenters (Spar-IBP)
# ---------------------------------------------------------------------------

class Barycenter(C.Structure):
    _fields_ = [("n", C.c_int32), ("d", C.c_int32), ("n_measures", C.c_int32), ("x", C.c_void_p),
                ("b", C.c_void_p), ("w", C.c_void_p), ("cost_norm", C.c_int32), ("cost_scale", C.c_double),
                ("dtype", C.c_int32)]


def spar_ibp(x, bs, w, *, eps, s, tol=1e-9, max_iter=10000, dtype="f64", kdtype=None, seed=0x5EED, problem_id=0,
             cost_norm=COST_MAXNORM, cost_scale=1.0, sampler="element", check_every=0, workspace=None, device=None,
             raise_on_error=True):
    """Spar-IBP barycenter of the measures bs (M x n) on the shared support x
    (n x d) with weights w (summing to 1): IBP on the sketches of Eq. (pois)
    with Eq. (pij-ot) for a = 1/n, measure k drawn with problem id
    problem_id + k.  Returns q (iterate type) and the solve's counters."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    dt = torch.float64 if dtype == "f64" else torch.float32
    xd = _dev(x, dt, dev)
    if xd.dim() == 1:
        xd = xd.reshape(-1, 1).contiguous()
    bd = _dev(bs, dt, dev).reshape(-1, xd.shape[0]).contiguous()
    M, n = bd.shape
    wh = np.ascontiguousarray(np.asarray(w, np.float64).reshape(M))
    kd = kdtype or dtype
    B = Barycenter(n, xd.shape[1], M, _ptr(xd), _ptr(bd), wh.ctypes.data, int(cost_norm), float(cost_scale),
                   F64 if dtype == "f64" else F32)
    prm = make_params(eps, math.inf, s, tol, max_iter, check_every, STOP_RESIDUAL, seed, problem_id, kd,
                      sampler=sampler)
    L = lib()
    L.sps_ibp_workspace_bytes.argtypes = [C.c_void_p, C.c_void_p]
    L.sps_ibp_workspace_bytes.restype = C.c_size_t
    L.spar_ibp.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p]
    L.spar_ibp.restype = C.c_int
    nbytes = L.sps_ibp_workspace_bytes(C.byref(B), C.byref(prm))
    if nbytes == 0:
        raise SpsError(SPS_ERR_INVALID_ARG, last_error())
    ws = _workspace(nbytes, dev, workspace)
    q = torch.empty(n, dtype=torch.float64 if kd == "f64" else torch.float32, device=dev)
    res = Result()
    st = L.spar_ibp(C.byref(B), C.byref(prm), _ptr(ws), nbytes, _ptr(q), C.byref(res), _stream())
    if raise_on_error:
        _check(st)
    out = res.as_dict()
    out["status_code"] = st
    out["q"] = q
    out["workspace"] = ws
    return out


# ---------------------------------------------------------------------------
# batches of problems over shared point sets
# ---------------------------------------------------------------------------

_side_streams = {}


def _side_stream(dev):
    if dev not in _side_streams:
        _side_streams[dev] = torch.cuda.Stream(dev)
    return _side_streams[dev]


class Batch(C.Structure):
    _fields_ = [("n_sets", C.c_int32), ("d", C.c_int32), ("set_off", C.c_void_p), ("pts", C.c_void_p),
                ("mass", C.c_void_p), ("n_pairs", C.c_int32), ("src", C.c_void_p), ("dst", C.c_void_p),
                ("s", C.c_void_p), ("cost_norm", C.c_int32), ("cost_scale", C.c_double), ("dtype", C.c_int32)]


class BatchOpts(C.Structure):
    _fields_ = [("lanes_per_row", C.c_int32), ("block_threads", C.c_int32), ("use_graph", C.c_int32),
                ("chosen_lanes", C.c_int32), ("chosen_threads", C.c_int32), ("tune_ms", C.c_float)]


def spar_sink_batched(sets, pairs, s, *, eps, lam=math.inf, tol=1e-5, max_iter=1000, dtype="f32", kdtype=None,
                      seed=0x5EED, problem_id=0, cost_norm=COST_MAXNORM, cost_scale=1.0, absorb_tau=0.0,
                      lanes_per_row=0, block_threads=0, use_graph=0, init_alpha=None, init_beta=None,
                      workspace=None, device=None, raise_on_error=True, sampler="element"):
    """Every pair (src, dst) of `pairs` solved as Alg. 3 (lam = inf) or Alg. 4
    on the sets `sets` = [(points k x d, masses k), ...] with budget s[p] and
    Philox problem id problem_id + p; sampler "element" (one decision per
    element) or "skip" (geometric gaps with thinning), each pair's sketch the
    one a single solve with its problem id draws.  Returns the per-pair results, the
    potentials split per pair, and the launch shape the library used."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    dt = torch.float64 if dtype == "f64" else torch.float32
    pts = torch.cat([torch.as_tensor(p, dtype=dt).reshape(len(m), -1) for p, m in sets]).to(dev).contiguous()
    mass = torch.cat([torch.as_tensor(m, dtype=dt).reshape(-1) for _, m in sets]).to(dev).contiguous()
    d = int(pts.shape[1])
    set_off = np.zeros(len(sets) + 1, np.int64)
    set_off[1:] = np.cumsum([len(m) for _, m in sets])
    src = np.ascontiguousarray([p[0] for p in pairs], np.int32)
    dst = np.ascontiguousarray([p[1] for p in pairs], np.int32)
    sv = np.ascontiguousarray(np.broadcast_to(np.asarray(s, np.float64), (len(pairs),)))
    bt = Batch(len(sets), d, set_off.ctypes.data, _ptr(pts), _ptr(mass), len(pairs), src.ctypes.data,
               dst.ctypes.data, sv.ctypes.data, int(cost_norm), float(cost_scale), DTYPE_CODES[dtype])
    kd = kdtype or ("f32" if dtype == "f64" else dtype)
    ia, ib = _dev(init_alpha, torch.float32, dev), _dev(init_beta, torch.float32, dev)
    prm = make_params(eps, lam, 1.0, tol, max_iter, 0, STOP_RESIDUAL, seed, problem_id, kd, 1, absorb_tau, ia, ib,
                      sampler=sampler)
    L = lib()
    L.sps_batch_workspace_bytes.argtypes = [C.c_void_p, C.c_void_p]
    L.sps_batch_workspace_bytes.restype = C.c_size_t
    L.spar_sink_batched.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]
    L.spar_sink_batched.restype = C.c_int
    nbytes = L.sps_batch_workspace_bytes(C.byref(bt), C.byref(prm))
    if nbytes == 0:
        raise SpsError(SPS_ERR_INVALID_ARG, last_error())
    ws = _workspace(nbytes, dev, workspace)
    sizes = np.diff(set_off)
    n_tot = int(sum(sizes[p[0]] for p in pairs))
    m_tot = int(sum(sizes[p[1]] for p in pairs))
    alpha = torch.empty(n_tot, dtype=torch.float32, device=dev)
    beta = torch.empty(m_tot, dtype=torch.float32, device=dev)
    opts = BatchOpts(int(lanes_per_row), int(block_threads), int(use_graph), 0, 0, 0.0)
    res = (Result * len(pairs))()
    cur = torch.cuda.current_stream(dev)
    side = None
    if use_graph and cur.cuda_stream == 0:
        # graph capture needs a stream other than the legacy default stream
        side = _side_stream(dev)
        side.wait_stream(cur)
    stream = C.c_void_p((side or cur).cuda_stream)
    st = L.spar_sink_batched(C.byref(bt), C.byref(prm), C.byref(opts), _ptr(ws), nbytes, _ptr(alpha), _ptr(beta),
                             C.byref(res), stream)
    if side is not None:
        cur.wait_stream(side)
    if raise_on_error:
        _check(st)
    ro = np.concatenate([[0], np.cumsum([sizes[p[0]] for p in pairs])])
    co = np.concatenate([[0], np.cumsum([sizes[p[1]] for p in pairs])])
    return {"status_code": st, "results": [r.as_dict() for r in res],
            "alpha": [alpha[ro[k]:ro[k + 1]] for k in range(len(pairs))],
            "beta": [beta[co[k]:co[k + 1]] for k in range(len(pairs))],
            "lanes_per_row": opts.chosen_lanes, "block_threads": opts.chosen_threads, "tune_ms": opts.tune_ms,
            "workspace": ws, "alpha_flat": alpha, "beta_flat": beta}


# ---------------------------------------------------------------------------
# learned warm start
# ---------------------------------------------------------------------------

class MlpInstance(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p), ("n", C.c_int32),
                ("m", C.c_int32), ("d", C.c_int32), ("cost_max", C.c_double), ("eps", C.c_double)]


def _mlp_lib():
    L = lib()
    if not getattr(L, "_mlp_ready", False):
        V, S_ = C.c_void_p, C.c_size_t
        L.sps_mlp_param_count.argtypes = [C.c_int32]
        L.sps_mlp_param_count.restype = S_
        L.sps_mlp_workspace_bytes.argtypes = []
        L.sps_mlp_workspace_bytes.restype = S_
        L.sps_mlp_init.argtypes = [V, V, C.c_int32, C.c_uint64, V]
        L.sps_mlp_sync_bf16.argtypes = [V, V, C.c_int32, V]
        L.sps_cost_max.argtypes = [V, C.c_int32, V, C.c_int32, C.c_int32, V, V, V]
        L.sps_cost_max_workspace_bytes.argtypes = [C.c_int32, C.c_int32, C.c_int32]
        L.sps_cost_max_workspace_bytes.restype = S_
        L.sps_cost_max_ws.argtypes = [V, C.c_int32, V, C.c_int32, C.c_int32, V, V, S_, V]
        L.sps_mlp_infer.argtypes = [V, V, V, V, V, V]
        L.sps_mlp_gauge_fix.argtypes = [V, V, V, V, V]
        L.sps_mlp_grad.argtypes = [V, V, V, V, V, V, V, V, V]
        L.sps_mlp_adam.argtypes = [V, V, V, V, V, C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float, V]
        for f in ("sps_mlp_init", "sps_mlp_sync_bf16", "sps_cost_max", "sps_cost_max_ws", "sps_mlp_infer",
                  "sps_mlp_gauge_fix",
                  "sps_mlp_grad", "sps_mlp_adam"):
            getattr(L, f).restype = C.c_int
        L._mlp_ready = True
    return L


def mlp_param_count(d):
    return int(_mlp_lib().sps_mlp_param_count(int(d)))


def _mlp_ws(device):
    return torch.empty(int(_mlp_lib().sps_mlp_workspace_bytes()) + 256, dtype=torch.uint8, device=device)


def cost_max(x, y, device=None, full_sweep=False):
    """Exact maximum of the binary32 squared distances (the SPS_COST_MAXNORM
    divisor): by default through sps_cost_max_ws (the pruned search above 1e8
    pairs, in a workspace allocated here), or with full_sweep=True through
    sps_cost_max (every pair)."""
    dev = torch.device(device) if device is not None else (x.device if isinstance(x, torch.Tensor) and x.is_cuda
                                                           else torch.device("cuda"))
    xd = _dev(x, torch.float32, dev).contiguous()
    yd = _dev(y, torch.float32, dev).contiguous()
    out = C.c_double(0.0)
    L = _mlp_lib()
    n, m, d = xd.shape[0], yd.shape[0], xd.shape[1]
    if full_sweep:
        st = L.sps_cost_max(_ptr(xd), n, _ptr(yd), m, d, C.byref(out), _ptr(_mlp_ws(dev)), _stream())
    else:
        nbytes = L.sps_cost_max_workspace_bytes(n, m, d)
        if nbytes == 0:
            raise SpsError(SPS_ERR_INVALID_ARG, "bad cost_max sizes")
        ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        st = L.sps_cost_max_ws(_ptr(xd), n, _ptr(yd), m, d, C.byref(out), _ptr(ws), nbytes, _stream())
    _check(st, allow_not_converged=False)
    return out.value


def mlp_instance(x, a, y, b, cost_max_value, eps=1.0):
    """Device tensors and the C struct of one instance (kept alive together)."""
    inst = MlpInstance(_ptr(x), _ptr(y), _ptr(a), _ptr(b), x.shape[0], y.shape[0], x.shape[1],
                       float(cost_max_value), float(eps))
    inst.keep = (x, a, y, b)
    return inst


def mlp_init(params, params_bf16, d, seed):
    _check(_mlp_lib().sps_mlp_init(_ptr(params), _ptr(params_bf16), int(d), int(seed), _stream()), False)


def mlp_sync_bf16(params, params_bf16, d):
    _check(_mlp_lib().sps_mlp_sync_bf16(_ptr(params), _ptr(params_bf16), int(d), _stream()), False)


def mlp_infer(params_bf16, inst, alpha_out, beta_out, ws=None):
    ws = ws if ws is not None else _mlp_ws(alpha_out.device)
    _check(_mlp_lib().sps_mlp_infer(_ptr(params_bf16), C.byref(inst), _ptr(alpha_out), _ptr(beta_out), _ptr(ws),
                                    _stream()), False)


def mlp_gauge_fix(inst, alpha, beta, ws=None):
    ws = ws if ws is not None else _mlp_ws(alpha.device)
    _check(_mlp_lib().sps_mlp_gauge_fix(C.byref(inst), _ptr(alpha), _ptr(beta), _ptr(ws), _stream()), False)


def mlp_grad(params, params_bf16, inst, alpha_t, beta_t, grad, ws=None, want_loss=True):
    ws = ws if ws is not None else _mlp_ws(grad.device)
    loss = C.c_float(0.0)
    _check(_mlp_lib().sps_mlp_grad(_ptr(params), _ptr(params_bf16), C.byref(inst), _ptr(alpha_t), _ptr(beta_t),
                                   _ptr(grad), C.byref(loss) if want_loss else None, _ptr(ws), _stream()), False)
    return loss.value if want_loss else None


def mlp_adam(params, params_bf16, m1, m2, grad, d, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(_mlp_lib().sps_mlp_adam(_ptr(params), _ptr(params_bf16), _ptr(m1), _ptr(m2), _ptr(grad), int(d),
                                   int(step), float(lr), float(beta1), float(beta2), float(eps), _stream()), False)
