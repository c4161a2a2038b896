"""GPU checks of the learned warm start: cost divisor, inference, gradient and
Adam kernels against the FP64 CPU reference, and the iterations the trained
network saves on held-out instances (with the same final objective)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp_oracle as M  # noqa: E402
from paper_2306_06581_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_06581_gb300 import build, sparsink
    build.build()
    return sparsink


def _f32(z):
    return np.asarray(z, np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def inst_data():
    w = inputs.ot_gmm16(700, seed=11)
    x, y, a = _f32(w.x), _f32(w.y)[:500], _f32(w.a)
    b = _f32(w.b[:500] / w.b[:500].sum())
    cm = float(((x.astype(np.float32)[:, None] - y.astype(np.float32)[None]) ** 2).sum(-1).max())
    return x, a, y, b, cm


def test_cost_max_reproduces_maxnorm(S):
    w = inputs.ot_gmm16(3000, seed=12)
    x, y, a, b = _f32(w.x), _f32(w.y), _f32(w.a), _f32(w.b)
    cm = S.cost_max(torch.tensor(x, dtype=torch.float32, device="cuda"), torch.tensor(y, dtype=torch.float32, device="cuda"))
    ref = ((x.astype(np.float32)[:, None] - y.astype(np.float32)[None]) ** 2).sum(-1).max()
    assert abs(cm - float(ref)) <= 4e-7 * float(ref)
    kw = dict(eps=0.01, s=w.s, tol=1e-5, max_iter=5000, dtype="f32", seed=w.seed, log_domain=1)
    r1 = S.spar_sink_ot(a, b, x, y, **kw)
    r2 = S.spar_sink_ot(a, b, x, y, cost_norm=S.COST_SCALE, cost_scale=cm, **kw)
    assert r1["nnz"] == r2["nnz"] and r1["iters"] == r2["iters"] and r1["obj"] == r2["obj"]


@pytest.mark.parametrize("d", [3, 10])
def test_cost_max_pruned_equals_full_sweep(S, d):
    # above 1e8 pairs the workspace form evaluates only the pairs that can reach the maximum (grid cells
    # for d <= 4, radial bounds for d > 4); the maximum is the same binary32 value as every pair's
    n, m = 12000, 10000
    g = torch.Generator().manual_seed(40 + d)
    x = torch.randn(n, d, generator=g).cuda()
    y = (0.5 * torch.rand(m, d, generator=g) + 0.25).cuda()
    pruned = S.cost_max(x, y)
    full = S.cost_max(x, y, full_sweep=True)
    assert pruned == full
    ref = max(float(((x[i:i + 1000, None] - y[None]) ** 2).sum(-1).max()) for i in range(0, n, 1000))
    assert abs(pruned - ref) <= 4e-7 * ref


def test_inference_matches_reference(S, inst_data):
    from paper_2306_06581_gb300.warmstart import WarmStart
    x, a, y, b, cm = inst_data
    wts = inputs.mlp_weights(3, 21)
    net = WarmStart(3)
    net.set_weights(wts)
    al, be = net.predict(net.instance(x, a, y, b, cm))
    ra, rb = M.predict(wts, 3, x, a, y, b, cm)
    assert np.abs(al.cpu().numpy() - ra).max() <= 2e-5 * max(1.0, np.abs(ra).max())
    assert np.abs(be.cpu().numpy() - rb).max() <= 2e-5 * max(1.0, np.abs(rb).max())


def test_gradient_matches_reference(S, inst_data):
    from paper_2306_06581_gb300.warmstart import WarmStart
    x, a, y, b, cm = inst_data
    rng = np.random.default_rng(3)
    wts = inputs.mlp_weights(3, 22)
    ta = rng.normal(0, 0.05, len(a)); tb = rng.normal(0, 0.05, len(b))
    ta[5] = -np.inf
    eps = 0.05
    net = WarmStart(3)
    net.set_weights(wts)
    inst = net.instance(x, a, y, b, cm, eps)
    g = torch.zeros_like(net.w)
    loss = S.mlp_grad(net.w, net.wb, inst, torch.tensor(ta, dtype=torch.float32, device="cuda"),
                      torch.tensor(tb, dtype=torch.float32, device="cuda"), g)
    L, gr = M.loss_grad(wts, 3, x, a, y, b, cm, ta, tb, eps)
    assert abs(loss - L) <= 1e-4 * L
    gg = g.cpu().numpy().astype(np.float64)
    o = M.layout(3)
    n1 = o["size"]
    for side in (0, n1):
        for nm in ("We", "ce", "W1", "b1", "W2", "b2", "w3", "b3"):
            s0, sz = o[nm]
            ref = gr[side + s0: side + s0 + sz]
            got = gg[side + s0: side + s0 + sz]
            assert np.abs(got - ref).max() <= 2e-3 * max(np.abs(ref).max(), 1e-3), (side, nm)


def test_adam_matches_reference(S):
    from paper_2306_06581_gb300.warmstart import WarmStart
    net = WarmStart(3)
    n = net.w.numel()
    rng = np.random.default_rng(4)
    w0 = inputs.mlp_weights(3, 23)
    g = rng.normal(0, 1e-2, n).astype(np.float32).astype(np.float64)
    net.set_weights(w0)
    w, m1, m2 = w0.copy(), np.zeros(n), np.zeros(n)
    for t in (1, 2, 3):
        net.g.copy_(torch.tensor(g * t, dtype=torch.float32))
        S.mlp_adam(net.w, net.wb, net.m1, net.m2, net.g, 3, t, 1e-3)
        w, m1, m2 = M.adam(w, m1, m2, g * t, t, 1e-3)
    assert np.abs(net.w.cpu().numpy() - w).max() <= 1e-6


def test_warm_start_saves_iterations(S):
    from paper_2306_06581_gb300 import warmstart as WS
    # 128 training instances of the 16-component mixture family (n = 3000), 3000 Adam steps;
    # 8 held-out instances (measured on a GB300: about 11% fewer iterations)
    n = 3000
    data = []
    for k in range(128):
        w = inputs.ot_gmm16(n, seed=1000 + k)
        inst, al, be, _ = WS.solve_targets(w, 0.01, w.s, seed=w.seed)
        data.append((inst, al, be))
    net = WS.WarmStart(3, seed=5)
    losses = WS.train(net, data, 3000, lr=2e-3, lr_end=2e-4)
    assert np.mean(losses[-128:]) < 0.6 * np.mean(losses[:128])
    cold, warm = [], []
    for k in range(8):
        w = inputs.ot_gmm16(n, seed=2000 + k)
        t = lambda z: torch.tensor(_f32(z), dtype=torch.float32, device="cuda")
        x, y, a, b = t(w.x), t(w.y), t(w.a), t(w.b)
        cm = S.cost_max(x, y)
        kw = dict(eps=0.01, s=w.s, tol=1e-5, max_iter=20000, dtype="f32", seed=w.seed, log_domain=1,
                  cost_norm=S.COST_SCALE, cost_scale=cm)
        rc = S.spar_sink_ot(a, b, x, y, **kw)
        al, be = net.predict(net.instance(x, a, y, b, cm))
        rw = S.spar_sink_ot(a, b, x, y, init_alpha=al, init_beta=be, **kw)
        assert rc["status"] == 0 and rw["status"] == 0
        assert abs(rw["obj"] - rc["obj"]) <= 1e-4 * abs(rc["obj"])
        cold.append(rc["iters"]); warm.append(rw["iters"])
    print(f"held-out iterations: cold {cold} warm {warm}")
    assert np.mean(warm) <= 0.95 * np.mean(cold)
