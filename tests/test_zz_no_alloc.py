"""spar_sink_ot_noalloc: Spar-Sink OT for callers that cannot allocate device
memory at solve time (their device memory belongs to another allocator, or
they may only allocate at start-up) and therefore cannot supply the workspace
spar_sink_ot asks for.  The entry point uses a fixed static scratch array
inside the library instead.

Checked through the C ABI against spar_sink_ot with a caller workspace, which
runs the same deterministic kernels on the same inputs, so everything must
agree bit for bit (status, nnz, iterations, residual, objective terms and
both potentials):
  - two FP64 calls in a row;
  - a log-domain call right after a larger plain call (stale scratch from the
    bigger problem must not leak into the staging or absorption state);
  - an FP32 problem after the FP64 calls;
  - a warmed-up call changes neither torch's allocated bytes nor the device's
    free memory (no allocation of the call's own);
  - a problem larger than the scratch array is refused with SPS_ERR_WORKSPACE.
This file is collected last so that a failing run has already run the rest.
"""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_06581_gb300 import inputs  # noqa: E402

SCRATCH = 16 << 20


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_06581_gb300 import build, sparsink
    build.build()
    f = sparsink.lib().spar_sink_ot_noalloc
    f.argtypes = [C.c_void_p] * 6
    f.restype = C.c_int
    return sparsink


def _call_noalloc(S, M, prm, it_dtype, alpha=None, beta=None):
    dev = M.keep[0].device
    if alpha is None:
        alpha = torch.full((M.prob.n,), float("nan"), dtype=it_dtype, device=dev)
        beta = torch.full((M.prob.m,), float("nan"), dtype=it_dtype, device=dev)
    res = S.Result()
    st = S.lib().spar_sink_ot_noalloc(C.byref(M.prob), C.byref(prm), C.c_void_p(alpha.data_ptr()),
                                      C.c_void_p(beta.data_ptr()), C.byref(res),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, res.as_dict(), alpha, beta


_EXACT = ("status", "nnz", "iters", "residual", "obj", "obj_sparse", "transport", "neg_entropy", "logp", "mass",
          "kl_a", "kl_b", "unreach_a", "unreach_b", "n_absorb")


def _compare_exact(ref, got, alpha, beta):
    for k in _EXACT:
        assert got[k] == ref[k], (k, got[k], ref[k])
    ra, ga = ref["alpha"].cpu().numpy(), alpha.cpu().numpy()
    rb, gb = ref["beta"].cpu().numpy(), beta.cpu().numpy()
    # bit-equal, -inf (unreachable rows) included
    assert np.array_equal(ra.view(np.uint8), ga.view(np.uint8))
    assert np.array_equal(rb.view(np.uint8), gb.view(np.uint8))


def _gmm_f32(n, seed, eps):
    w = inputs.ot_gmm(n, d=3, k=8, seed=seed, eps=eps, s_factor=16.0)
    return w, tuple(np.asarray(z, np.float32) for z in (w.x, w.y, w.a, w.b))


def test_noalloc_matches_workspace_entry_point_twice(S):
    w = inputs.ot_n1000()
    kw = dict(eps=w.eps, s=w.s, tol=w.tol, max_iter=5000, dtype="f64", seed=w.seed)
    ref = S.spar_sink_ot(w.a, w.b, w.x, w.y, **kw)
    M = S.make_problem(w.a, w.b, w.x, w.y, dtype="f64")
    prm = S.make_params(w.eps, math.inf, w.s, w.tol, 5000, seed=w.seed, kdtype="f64")
    assert S.sps_workspace_bytes(M.prob, prm, S.OP_SPAR_SINK) <= SCRATCH
    for _ in range(2):
        st, got, alpha, beta = _call_noalloc(S, M, prm, torch.float64)
        assert st == S.SPS_OK, S.last_error()
        _compare_exact(ref, got, alpha, beta)


def test_noalloc_log_domain_after_larger_plain_call(S):
    # a larger plain FP32 solve fills more of the scratch array first
    wb, (xb, yb, ab, bb) = _gmm_f32(2200, seed=33, eps=0.1)
    Mb = S.make_problem(ab, bb, xb, yb, dtype="f32")
    pb = S.make_params(wb.eps, math.inf, wb.s, 1e-5, 20000, kdtype="f32")
    big = S.sps_workspace_bytes(Mb.prob, pb, S.OP_SPAR_SINK)
    st, gb, al_b, be_b = _call_noalloc(S, Mb, pb, torch.float32)
    assert st == S.SPS_OK, S.last_error()
    refb = S.spar_sink_ot(ab, bb, xb, yb, eps=wb.eps, s=wb.s, tol=1e-5, max_iter=20000, dtype="f32")
    _compare_exact(refb, gb, al_b, be_b)
    # then a smaller stabilised (log-domain, absorbing) solve at eps = 0.01
    ws_, (xs, ys, as_, bs) = _gmm_f32(1200, seed=34, eps=0.01)
    Ms = S.make_problem(as_, bs, xs, ys, dtype="f32")
    ps = S.make_params(ws_.eps, math.inf, ws_.s, 1e-5, 20000, kdtype="f32", log_domain=1)
    assert S.sps_workspace_bytes(Ms.prob, ps, S.OP_SPAR_SINK) < big
    st, got, alpha, beta = _call_noalloc(S, Ms, ps, torch.float32)
    assert st == S.SPS_OK, S.last_error()
    ref = S.spar_sink_ot(as_, bs, xs, ys, eps=ws_.eps, s=ws_.s, tol=1e-5, max_iter=20000, dtype="f32", log_domain=1)
    assert ref["n_absorb"] >= 1 or ref["iters"] >= 1
    _compare_exact(ref, got, alpha, beta)


def test_noalloc_after_other_problem(S):
    # a different, FP32 problem after the FP64 calls: stale scratch contents must not matter
    w, (x, y, a, b) = _gmm_f32(1500, seed=21, eps=0.05)
    ref = S.spar_sink_ot(a, b, x, y, eps=w.eps, s=w.s, tol=1e-5, max_iter=20000, dtype="f32")
    M = S.make_problem(a, b, x, y, dtype="f32")
    prm = S.make_params(w.eps, math.inf, w.s, 1e-5, 20000, kdtype="f32")
    st, got, alpha, beta = _call_noalloc(S, M, prm, torch.float32)
    assert st == S.SPS_OK, S.last_error()
    _compare_exact(ref, got, alpha, beta)


def test_noalloc_allocates_nothing(S):
    w = inputs.ot_n1000()
    M = S.make_problem(w.a, w.b, w.x, w.y, dtype="f64")
    prm = S.make_params(w.eps, math.inf, w.s, w.tol, 5000, seed=w.seed, kdtype="f64")
    need = S.sps_workspace_bytes(M.prob, prm, S.OP_SPAR_SINK)
    # a device allocation of the workspace's size maps at least 2 MiB, more than the slack below
    assert need > (2 << 20)
    alpha = torch.empty(M.prob.n, dtype=torch.float64, device=M.keep[0].device)
    beta = torch.empty_like(alpha[:M.prob.m])
    st, _, _, _ = _call_noalloc(S, M, prm, torch.float64, alpha, beta)   # warm-up: module and address set up
    assert st == S.SPS_OK, S.last_error()
    torch.cuda.synchronize()
    torch_before = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    st, _, _, _ = _call_noalloc(S, M, prm, torch.float64, alpha, beta)
    assert st == S.SPS_OK, S.last_error()
    free_after, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == torch_before
    # the call creates CUDA events (host-side objects); 1 MiB of slack covers any driver bookkeeping
    assert free_after >= free_before - (1 << 20), (free_before, free_after)


def test_noalloc_rejects_problem_larger_than_scratch(S):
    w = inputs.uot_n20000()
    M = S.make_problem(w.a, w.b, w.x, w.y, dtype="f32")
    prm = S.make_params(w.eps, math.inf, w.s, 1e-5, 100, kdtype="f32")
    assert S.sps_workspace_bytes(M.prob, prm, S.OP_SPAR_SINK) > SCRATCH
    st, got, alpha, beta = _call_noalloc(S, M, prm, torch.float32)
    assert st == S.SPS_ERR_WORKSPACE
    assert "spar_sink_ot" in S.last_error() and "scratch" in S.last_error()
    assert torch.isnan(alpha).all()   # nothing was written
