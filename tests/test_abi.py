"""The C ABI library loads and exports every entry point include/sparsink.h
declares; argument errors are rejected on the host before any launch (these
calls need no GPU)."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    from paper_2306_06581_gb300 import build, sparsink
    build.build()
    return sparsink


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "sizeof"):
                names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(S):
    lib = C.CDLL(S.LIB_PATH)
    declared = _declared_functions()
    assert {"sinkhorn_dense", "sparsify_kernel", "spar_sink_ot", "spar_sink_uot", "sps_workspace_bytes",
            "sps_last_error"} <= declared
    for name in declared:
        assert hasattr(lib, name), name


def _prob(S, n=100, m=120, d=3, dtype=1):
    fake = C.c_void_p(256)
    return S.Problem(n, m, d, fake, fake, None, 1, 1.0, fake, fake, dtype)


def test_workspace_sizes(S):
    P = _prob(S)
    Q = S.make_params(0.1, math.inf, 5000.0, kdtype="f32")
    sp, it, de = (S.sps_workspace_bytes(P, Q, op) for op in (0, 1, 2))
    assert 0 < de and 0 < sp < it
    # capacity grows with s and values with their width
    Q2 = S.make_params(0.1, math.inf, 10000.0, kdtype="f32")
    assert S.sps_workspace_bytes(P, Q2, 1) > it
    Q3 = S.make_params(0.1, math.inf, 5000.0, kdtype="f64")
    assert S.sps_workspace_bytes(P, Q3, 1) > it


@pytest.mark.parametrize("kw,frag", [
    (dict(eps=-1.0), "eps"), (dict(eps=float("nan")), "eps"), (dict(s=0.0), "budget"),
    (dict(lam=0.0), "lambda"), (dict(max_iter=0), "max_iter"), (dict(tol=-1.0), "tol"),
])
def test_invalid_params_rejected(S, kw, frag):
    P = _prob(S)
    base = dict(eps=0.1, lam=math.inf, s=1000.0, tol=1e-6, max_iter=10)
    base.update(kw)
    Q = S.make_params(base["eps"], base["lam"], base["s"], base["tol"], base["max_iter"])
    assert S.sps_workspace_bytes(P, Q, 1) == 0
    assert frag in S.last_error()


def test_sampler_and_modes_validated(S):
    P = _prob(S)
    Q = S.make_params(0.1, math.inf, 1000.0, sampler=2)
    assert S.sps_workspace_bytes(P, Q, 1) == 0
    assert "sampler" in S.last_error()
    Q = S.make_params(0.1, math.inf, 1000.0, sketch_mode=5)
    assert S.sps_workspace_bytes(P, Q, 1) == 0
    assert "sketch_mode" in S.last_error()
    # the skip sampler needs no padded single-pass slots: its workspace is smaller
    big = _prob(S, n=4000, m=4000)
    el = S.sps_workspace_bytes(big, S.make_params(0.1, math.inf, 2e5, sampler="element"), 1)
    sk = S.sps_workspace_bytes(big, S.make_params(0.1, math.inf, 2e5, sampler="skip"), 1)
    assert 0 < sk < el
    # both samplers for UOT as well
    assert S.sps_workspace_bytes(big, S.make_params(0.1, 1.0, 2e5, sampler="skip"), 1) > 0


def test_invalid_problem_rejected(S):
    Q = S.make_params(0.1, math.inf, 1000.0)
    assert S.sps_workspace_bytes(_prob(S, n=0), Q, 1) == 0
    assert S.sps_workspace_bytes(_prob(S, dtype=3), Q, 1) == 0
    P = _prob(S)
    P.x = None
    assert S.sps_workspace_bytes(P, Q, 1) == 0
    res = S.Result()
    # a null workspace is refused before any launch
    assert S.lib().spar_sink_ot(C.byref(_prob(S)), C.byref(Q), None, 0, None, None, C.byref(res), None) == S.SPS_ERR_INVALID_ARG
    # OT entry with finite lambda, UOT entry with infinite lambda
    Qu = S.make_params(0.1, 1.0, 1000.0)
    assert S.lib().spar_sink_ot(C.byref(_prob(S)), C.byref(Qu), C.c_void_p(256), 1 << 40, None, None, C.byref(res), None) == S.SPS_ERR_INVALID_ARG
    assert S.lib().spar_sink_uot(C.byref(_prob(S)), C.byref(Q), C.c_void_p(256), 1 << 40, None, None, C.byref(res), None) == S.SPS_ERR_INVALID_ARG
    # a workspace smaller than required
    assert S.lib().spar_sink_ot(C.byref(_prob(S)), C.byref(Q), C.c_void_p(256), 16, None, None, C.byref(res), None) == S.SPS_ERR_WORKSPACE


def test_binding_fails_loudly_without_library(S, tmp_path, monkeypatch):
    monkeypatch.setattr(S, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(S, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        S.lib()


def test_iteration_controls_validated(S):
    P = _prob(S)
    Q = S.make_params(0.1, math.inf, 1000.0, check_every=-3)
    assert S.sps_workspace_bytes(P, Q, 1) == 0
    assert "check_every" in S.last_error()
    assert S.sps_workspace_bytes(P, S.make_params(0.1, math.inf, 1000.0, check_every=0), 1) > 0
    for tau in (float("nan"), math.inf, -1.0):
        Q = S.make_params(0.01, math.inf, 1000.0, kdtype="f32", log_domain=1, absorb_tau=tau)
        assert S.sps_workspace_bytes(P, Q, 1) == 0, tau
        assert "absorb_tau" in S.last_error()
    assert S.sps_workspace_bytes(P, S.make_params(0.01, math.inf, 1000.0, kdtype="f32", log_domain=1,
                                                  absorb_tau=20.0), 1) > 0


def _batch(S, sets=(100, 120, 80), pairs=((0, 1), (1, 2), (2, 0)), s=None, d=2, cost_norm=1, cost_scale=1.0,
           dtype=1):
    import numpy as np
    off = np.concatenate([[0], np.cumsum(sets)]).astype(np.int64)
    src = np.array([p[0] for p in pairs], np.int32)
    dst = np.array([p[1] for p in pairs], np.int32)
    sb = np.array(s if s is not None else [1000.0] * len(pairs), np.float64)
    B = S.Batch(len(sets), d, off.ctypes.data, 256, 256, len(pairs), src.ctypes.data, dst.ctypes.data,
                sb.ctypes.data, cost_norm, cost_scale, dtype)
    return B, (off, src, dst, sb)


def _batch_bytes(S, B, Q):
    f = S.lib().sps_batch_workspace_bytes
    f.argtypes = [C.c_void_p, C.c_void_p]
    f.restype = C.c_size_t
    return int(f(C.byref(B), C.byref(Q)))


def test_batch_arguments_validated(S):
    # spar_sink_batched's host-side checks, through its workspace-size call (no GPU needed)
    Q = S.make_params(0.01, 1.0, 1.0, 1e-5, 100, kdtype="f32")
    B, keep = _batch(S)
    ok = _batch_bytes(S, B, Q)
    assert ok > 0
    # the workspace grows with the budgets
    B2, keep2 = _batch(S, s=[4000.0] * 3)
    assert _batch_bytes(S, B2, Q) > ok
    bad = [
        (dict(d=0), "d"), (dict(d=17), "d"),
        (dict(sets=(100, 0, 80)), "empty"),
        (dict(pairs=((0, 1), (1, 3))), "out of range"), (dict(pairs=((0, 1), (-1, 2))), "out of range"),
        (dict(s=[1000.0, 0.0, 1000.0]), "budget"), (dict(s=[1000.0, float("nan"), 1000.0]), "budget"),
        (dict(sets=(20000, 10000), pairs=((0, 1),)), "shared memory"),   # 2 n + m = 50000 > 49152
        (dict(cost_norm=2, cost_scale=math.inf), "cost_scale"), (dict(cost_norm=2, cost_scale=0.0), "cost_scale"),
        (dict(cost_norm=5), "cost_norm"), (dict(dtype=2), "F32 or F64"),
    ]
    for kw, frag in bad:
        Bb, kb = _batch(S, **kw)
        assert _batch_bytes(S, Bb, Q) == 0, kw
        assert frag in S.last_error(), (kw, S.last_error())
    # 2 n + m at the limit is accepted
    Bl, kl = _batch(S, sets=(16384, 16384), pairs=((0, 1),))
    assert _batch_bytes(S, Bl, Q) > 0
    # both samplers
    assert _batch_bytes(S, B, S.make_params(0.01, 1.0, 1.0, 1e-5, 100, kdtype="f32", sampler="skip")) > 0
    # parameters the batched solver does not take
    for Qb, frag in [(S.make_params(0.01, 1.0, 1.0, 1e-5, 100, kdtype="f64"), "F32, BF16 or F16"),
                     (S.make_params(0.01, 1.0, 1.0, 1e-5, 100, kdtype="f32", sampler=2), "sampler"),
                     (S.make_params(0.01, 1.0, 1.0, 1e-5, 100, kdtype="f32", stop_rule=1), "residual"),
                     (S.make_params(0.01, 1.0, 1.0, 1e-5, 0, kdtype="f32"), "max_iter"),
                     (S.make_params(0.0, 1.0, 1.0, 1e-5, 100, kdtype="f32"), "eps"),
                     (S.make_params(0.01, 1.0, 1.0, 1e-5, 100, kdtype="f32", absorb_tau=math.inf), "absorb_tau"),
                     (S.make_params(0.01, 1.0, 1.0, 1e-5, 100, kdtype="f32", absorb_tau=float("nan")), "absorb_tau")]:
        assert _batch_bytes(S, B, Qb) == 0, frag
        assert frag in S.last_error(), (frag, S.last_error())


def test_warm_start_arguments_validated(S):
    # the warm-start calls refuse bad arguments before any launch (fake device pointers are never touched)
    L = S._mlp_lib()
    f = C.c_void_p(256)
    assert S.mlp_param_count(0) == 0 and S.mlp_param_count(17) == 0 and S.mlp_param_count(3) > 0
    good = dict(lr=1e-3, b1=0.9, b2=0.999, eps=1e-8)
    for k, v in [("lr", float("nan")), ("lr", -1e-3), ("lr", math.inf), ("b1", 1.0), ("b1", -0.1),
                 ("b2", 1.0), ("b2", float("nan")), ("eps", 0.0), ("eps", math.inf)]:
        a = dict(good, **{k: v})
        st = L.sps_mlp_adam(f, f, f, f, f, 3, 1, a["lr"], a["b1"], a["b2"], a["eps"], None)
        assert st == S.SPS_ERR_INVALID_ARG, (k, v)
        assert "Adam" in S.last_error()
    assert L.sps_mlp_adam(f, f, f, f, f, 3, 0, 1e-3, 0.9, 0.999, 1e-8, None) == S.SPS_ERR_INVALID_ARG   # step 0
    assert L.sps_mlp_adam(f, f, f, f, f, 17, 1, 1e-3, 0.9, 0.999, 1e-8, None) == S.SPS_ERR_INVALID_ARG  # d > 16
    # instances: sizes, dimension, cost divisor and (for the gradient) the loss scale
    def inst(**kw):
        base = dict(x=256, y=256, a=256, b=256, n=10, m=12, d=3, cost_max=2.0, eps=0.1)
        base.update(kw)
        return S.MlpInstance(base["x"], base["y"], base["a"], base["b"], base["n"], base["m"], base["d"],
                             base["cost_max"], base["eps"])
    for kw in (dict(n=0), dict(d=17), dict(cost_max=0.0), dict(cost_max=math.inf), dict(x=None)):
        assert L.sps_mlp_infer(f, C.byref(inst(**kw)), f, f, f, None) == S.SPS_ERR_INVALID_ARG, kw
    for e in (0.0, math.inf, float("nan")):
        st = L.sps_mlp_grad(f, f, C.byref(inst(eps=e)), f, f, f, None, f, None)
        assert st == S.SPS_ERR_INVALID_ARG, e
        assert "eps" in S.last_error()
    assert L.sps_cost_max(f, 0, f, 5, 3, f, f, None) == S.SPS_ERR_INVALID_ARG
    # the workspace form: sizes, then a workspace below the required size, refused before any launch
    wb = L.sps_cost_max_workspace_bytes
    assert wb(0, 5, 3) == 0 and wb(5, 5, 0) == 0 and wb(5, 5, 17) == 0
    small, big3, big10 = wb(100, 100, 3), wb(20000, 20000, 3), wb(20000, 20000, 10)
    assert 0 < small < big3 and 0 < small < big10      # the pruned search's scratch only above 1e8 pairs
    assert L.sps_cost_max_ws(f, 100, f, 100, 3, f, f, small - 1, None) == S.SPS_ERR_WORKSPACE
    assert "workspace" in S.last_error()
    assert L.sps_cost_max_ws(f, 100, f, 0, 3, f, f, small, None) == S.SPS_ERR_INVALID_ARG
    assert L.sps_cost_max_ws(None, 100, f, 100, 3, f, f, small, None) == S.SPS_ERR_INVALID_ARG


def test_noalloc_refusals_need_no_device(S):
    # spar_sink_ot_noalloc refuses bad arguments and problems larger than its fixed scratch array on the
    # host, before it looks up the array or launches anything
    f = S.lib().spar_sink_ot_noalloc
    f.argtypes = [C.c_void_p] * 6
    f.restype = C.c_int
    res = S.Result()
    out = C.c_void_p(256)
    big = _prob(S, n=20000, m=20000, d=10)
    Q = S.make_params(0.05, math.inf, 3.17e6, kdtype="f32")
    assert S.sps_workspace_bytes(big, Q, 1) > 16 << 20
    assert f(C.byref(big), C.byref(Q), out, out, C.byref(res), None) == S.SPS_ERR_WORKSPACE
    assert "scratch" in S.last_error() and "spar_sink_ot" in S.last_error()
    Qbad = S.make_params(-1.0, math.inf, 1000.0)
    assert f(C.byref(_prob(S)), C.byref(Qbad), out, out, C.byref(res), None) == S.SPS_ERR_INVALID_ARG
    assert "eps" in S.last_error()


def test_barrier_selftest_refusals_need_no_device(S):
    f = S.lib().sps_selftest_barrier_timeout
    f.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    ms = C.c_float(0.0)
    assert f(None, 4096, C.byref(ms), None) == S.SPS_ERR_INVALID_ARG
    assert f(C.c_void_p(256), 4096, None, None) == S.SPS_ERR_INVALID_ARG
    assert f(C.c_void_p(256), 64, C.byref(ms), None) == S.SPS_ERR_WORKSPACE
    assert "workspace" in S.last_error()


def test_every_declaration_is_documented():
    # each entry point in include/*.h carries its own comment (meaning, layout, ownership, errors)
    seen = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        lines = open(os.path.join(ROOT, "include", fn)).read().split("\n")
        for k, line in enumerate(lines):
            m = re.match(r"^(?:const\s+)?(?:size_t|sps_status|const char\*|char\*)\s+([a-z_][a-z0-9_]*)\s*\(", line)
            if not m:
                continue
            above = "\n".join(lines[max(0, k - 3):k])
            assert "*/" in above, f"{fn}: {m.group(1)} has no comment above its declaration"
            seen.add(m.group(1))
    assert seen == _declared_functions()


def _wfr_prob(S, eta=0.5, cost_norm=0, with_C=False, kind=1):
    fake = C.c_void_p(256)
    return S.Problem(100, 120, 3, fake, fake, fake if with_C else None, cost_norm, 1.0, fake, fake, 1, kind, eta)


@pytest.mark.parametrize("kw,frag", [
    (dict(kind=7), "cost_kind"), (dict(eta=0.0), "eta"), (dict(eta=float("inf")), "eta"),
    (dict(eta=float("nan")), "eta"), (dict(cost_norm=1), "cost_norm"), (dict(with_C=True), "points"),
])
def test_wfr_arguments_validated(S, kw, frag):
    Q = S.make_params(0.1, 1.0, 1000.0)
    assert S.sps_workspace_bytes(_wfr_prob(S, **kw), Q, 1) == 0
    assert frag in S.last_error()


def test_wfr_accepted_for_the_sketch_and_refused_by_dense(S):
    Q = S.make_params(0.1, 1.0, 1000.0)
    assert S.sps_workspace_bytes(_wfr_prob(S), Q, 0) > 0
    assert S.sps_workspace_bytes(_wfr_prob(S), Q, 1) > 0
    assert S.sps_workspace_bytes(_wfr_prob(S), Q, 2) == 0
    assert "dense" in S.last_error()


def test_probs_validated(S):
    P = _prob(S)
    assert S.sps_workspace_bytes(P, S.make_params(0.1, 1.0, 1000.0, probs=2), 1) == 0
    assert "probs" in S.last_error()
    for probs in ("paper", "equal"):
        assert S.sps_workspace_bytes(P, S.make_params(0.1, 1.0, 1000.0, probs=probs), 1) > 0


def test_batch_refuses_equal_probabilities(S):
    Q = S.make_params(0.01, 1.0, 1.0, 1e-5, 100, kdtype="f32", probs="equal")
    B, keep = _batch(S)
    assert _batch_bytes(S, B, Q) == 0
    assert "probs" in S.last_error()


def _bary(S, n=50, M=3, w=None, d=1, dtype=1):
    import numpy as np
    wh = np.ascontiguousarray(np.asarray(w if w is not None else [1.0 / max(M, 1)] * max(M, 1), np.float64))
    fake = C.c_void_p(256)
    return S.Barycenter(n, d, M, fake, fake, wh.ctypes.data, 1, 1.0, dtype), wh


def _ibp_bytes(S, B, Q):
    f = S.lib().sps_ibp_workspace_bytes
    f.argtypes = [C.c_void_p, C.c_void_p]
    f.restype = C.c_size_t
    return int(f(C.byref(B), C.byref(Q)))


def test_ibp_arguments_validated(S):
    Q = S.make_params(0.05, math.inf, 500.0, 1e-9, 100, kdtype="f64")
    B, keep = _bary(S)
    assert _ibp_bytes(S, B, Q) > 0
    for kw, frag in ((dict(M=0), "n_measures"), (dict(M=65), "n_measures"), (dict(w=[0.5, 0.6, -0.1]), "w[2]"),
                     (dict(w=[0.2, 0.2, 0.2]), "sum to 1"), (dict(n=0), "support"), (dict(dtype=2), "dtype")):
        B, keep = _bary(S, **kw)
        assert _ibp_bytes(S, B, Q) == 0, kw
        assert frag in S.last_error(), (kw, S.last_error())
    B, keep = _bary(S)
    for q, frag in ((S.make_params(0.05, 1.0, 500.0, kdtype="f64"), "lambda"),
                    (S.make_params(0.05, math.inf, 500.0, kdtype="f32", log_domain=1), "log_domain"),
                    (S.make_params(0.05, math.inf, 500.0, probs="equal"), "probs"),
                    (S.make_params(-1.0, math.inf, 500.0), "eps")):
        assert _ibp_bytes(S, B, q) == 0
        assert frag in S.last_error(), (frag, S.last_error())
