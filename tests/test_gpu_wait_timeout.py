"""Failure detection without a GPU fault: the bounded wait of the iteration
kernels' grid barrier gives up, the device records it, the host reports it,
and the CUDA context stays usable.

sps_selftest_barrier_timeout runs the real barrier on two blocks, one of
which never arrives (a count that nothing completes), so the other block's
wait must run out after its fixed number of polls.  The check reads the
status through the C ABI, then runs an ordinary solve on the same device
and stream and compares it with the oracle.
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
    f = sparsink.lib().sps_selftest_barrier_timeout
    f.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return sparsink


def test_barrier_wait_times_out_and_context_survives(S, orc):
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    ms = C.c_float(0.0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = S.lib().sps_selftest_barrier_timeout(C.c_void_p(ws.data_ptr()), 4096, C.byref(ms), stream)
    assert st == S.SPS_ERR_CUDA, (st, S.last_error())
    assert "timed out" in S.last_error()
    assert ms.value > 0.0
    print(f"bounded barrier wait gave up after {ms.value:.0f} ms")
    # the context is intact: the same solve as the FP32 parity test, right after it, matches the oracle
    w = inputs.ot_gmm(3000, d=3, k=8, seed=11, eps=0.05, s_factor=16.0)
    f = lambda z: np.asarray(z, np.float32).astype(np.float64)
    x, y, a, b = f(w.x), f(w.y), f(w.a), f(w.b)
    g = S.spar_sink_ot(a, b, x, y, eps=w.eps, s=w.s, tol=1e-5, max_iter=20000, dtype="f32")
    o = orc.spar_sink(orc.OracleProblem(a, b, w.eps, w.s, math.inf, x=x, y=y), tol=1e-5, max_iter=20000)
    assert g["nnz"] == o["sketch"]["nnz"]
    assert g["status"] == o["info"]["status"] == 0
    assert abs(g["obj"] - o["obj"]) <= 1e-5 * abs(o["obj"])
