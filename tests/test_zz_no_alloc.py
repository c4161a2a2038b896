"""spar_sink_ot_noalloc: Spar-Sink OT for callers that cannot allocate device
memory at solve time (their device memory belongs to another allocator, or
they may only allocate at start-up) and therefore cannot supply the workspace
spar_sink_ot asks for.  The entry point uses a fixed static scratch array
inside the library instead.

Checked through the C ABI: two calls in a row give the same output as
spar_sink_ot with a caller workspace (within the FP64 tolerances of the
parity tests), a call on a different problem after them still agrees, and a
problem larger than the scratch array is refused with SPS_ERR_WORKSPACE.
This file is collected last so that a failing run has already run the rest.
"""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_06581_gb300 import inputs  # noqa: E402


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


def _call_noalloc(S, M, prm, it_dtype):
    dev = M.keep[0].device
    alpha = torch.full((M.prob.n,), float("nan"), dtype=it_dtype, device=dev)
    beta = torch.full((M.prob.m,), float("nan"), dtype=it_dtype, device=dev)
    res = S.Result()
    st = S.lib().spar_sink_ot_noalloc(C.byref(M.prob), C.byref(prm), C.c_void_p(alpha.data_ptr()),
                                      C.c_void_p(beta.data_ptr()), C.byref(res),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, res.as_dict(), alpha, beta


def _compare(ref, got, alpha, beta, atol):
    assert got["status"] == ref["status"] == 0
    assert got["nnz"] == ref["nnz"]
    assert abs(got["iters"] - ref["iters"]) <= 1
    assert abs(got["obj"] - ref["obj"]) <= 1e-8 * abs(ref["obj"])
    assert abs(got["obj_sparse"] - ref["obj_sparse"]) <= 1e-8 * abs(ref["obj_sparse"])
    if got["iters"] == ref["iters"]:
        ra, ga = ref["alpha"].cpu().numpy(), alpha.cpu().numpy()
        rb, gb = ref["beta"].cpu().numpy(), beta.cpu().numpy()
        fa, fb = np.isfinite(ra), np.isfinite(rb)
        assert np.array_equal(fa, np.isfinite(ga)) and np.array_equal(fb, np.isfinite(gb))
        assert np.abs(ra[fa] - ga[fa]).max() <= atol
        assert np.abs(rb[fb] - gb[fb]).max() <= atol


def test_noalloc_matches_workspace_entry_point_twice(S):
    w = inputs.ot_n1000()
    kw = dict(eps=w.eps, s=w.s, tol=w.tol, max_iter=5000, dtype="f64", seed=w.seed)
    ref = S.spar_sink_ot(w.a, w.b, w.x, w.y, **kw)
    M = S.make_problem(w.a, w.b, w.x, w.y, dtype="f64")
    prm = S.make_params(w.eps, math.inf, w.s, w.tol, 5000, seed=w.seed, kdtype="f64")
    assert S.sps_workspace_bytes(M.prob, prm, S.OP_SPAR_SINK) <= 16 << 20
    for _ in range(2):
        st, got, alpha, beta = _call_noalloc(S, M, prm, torch.float64)
        assert st == S.SPS_OK, S.last_error()
        _compare(ref, got, alpha, beta, atol=1e-9)


def test_noalloc_after_other_problem(S):
    # a different, FP32 problem after the FP64 calls: stale scratch contents must not matter
    w = inputs.ot_gmm(1500, d=3, k=8, seed=21, eps=0.05, s_factor=16.0)
    x, y, a, b = (np.asarray(z, np.float32) for z in (w.x, w.y, w.a, w.b))
    ref = S.spar_sink_ot(a, b, x, y, eps=w.eps, s=w.s, tol=1e-5, max_iter=20000, dtype="f32")
    M = S.make_problem(a, b, x, y, dtype="f32")
    prm = S.make_params(w.eps, math.inf, w.s, 1e-5, 20000, kdtype="f32")
    st, got, alpha, beta = _call_noalloc(S, M, prm, torch.float32)
    assert st == S.SPS_OK, S.last_error()
    assert got["nnz"] == ref["nnz"] and got["iters"] == ref["iters"]
    assert abs(got["obj"] - ref["obj"]) <= 1e-5 * abs(ref["obj"])


def test_noalloc_rejects_problem_larger_than_scratch(S):
    w = inputs.uot_n20000()
    M = S.make_problem(w.a, w.b, w.x, w.y, dtype="f32")
    prm = S.make_params(w.eps, math.inf, w.s, 1e-5, 100, kdtype="f32")
    assert S.sps_workspace_bytes(M.prob, prm, S.OP_SPAR_SINK) > 16 << 20
    st, got, alpha, beta = _call_noalloc(S, M, prm, torch.float32)
    assert st == S.SPS_ERR_WORKSPACE
    assert "spar_sink_ot" in S.last_error() and "scratch" in S.last_error()
    assert torch.isnan(alpha).all()   # nothing was written
