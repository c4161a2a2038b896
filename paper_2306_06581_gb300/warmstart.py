"""Training and use of the learned warm start (host orchestration only: every
forward, backward and optimiser step runs in the library's CUDA kernels).

Targets are the potentials that Spar-Sink itself returns on seeded training
instances (stabilised iterations, cost divisor from sps_cost_max_ws), with the
OT gauge fixed (sum a alpha = sum b beta).  A trained WarmStart predicts
starting potentials for sps_params.init_alpha / init_beta.
"""
from __future__ import annotations

import math

import torch

from . import sparsink as S


class WarmStart:
    def __init__(self, d=3, seed=1, device=None):
        self.dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.d = d
        n = S.mlp_param_count(d)
        self.w = torch.empty(n, dtype=torch.float32, device=self.dev)
        self.wb = torch.empty(n, dtype=torch.bfloat16, device=self.dev)
        self.m1 = torch.zeros(n, dtype=torch.float32, device=self.dev)
        self.m2 = torch.zeros(n, dtype=torch.float32, device=self.dev)
        self.g = torch.zeros(n, dtype=torch.float32, device=self.dev)
        self.ws = S._mlp_ws(self.dev)
        self.step = 0
        S.mlp_init(self.w, self.wb, d, seed)

    def set_weights(self, w):
        self.w.copy_(torch.as_tensor(w, dtype=torch.float32))
        S.mlp_sync_bf16(self.w, self.wb, self.d)

    def instance(self, x, a, y, b, cmax, eps=1.0):
        t = lambda z: S._dev(z, torch.float32, self.dev).contiguous()
        return S.mlp_instance(t(x), t(a), t(y), t(b), cmax, eps)

    def predict(self, inst):
        al = torch.empty(inst.n, dtype=torch.float32, device=self.dev)
        be = torch.empty(inst.m, dtype=torch.float32, device=self.dev)
        S.mlp_infer(self.wb, inst, al, be, self.ws)
        return al, be

    def train_step(self, inst, alpha_t, beta_t, lr):
        loss = S.mlp_grad(self.w, self.wb, inst, alpha_t, beta_t, self.g, self.ws)
        self.step += 1
        S.mlp_adam(self.w, self.wb, self.m1, self.m2, self.g, self.d, self.step, lr)
        return loss


def solve_targets(w, eps, s, tol=1e-5, max_iter=20000, seed=0x5EED, kdtype="f32", sampler="element"):
    """Spar-Sink on one instance; returns the instance's device tensors, the
    cost divisor and the gauge-fixed potentials (the training targets)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    t = lambda z: torch.as_tensor(z, dtype=torch.float32).to(dev).contiguous()
    x, y, a, b = t(w.x), t(w.y), t(w.a), t(w.b)
    cm = S.cost_max(x, y)
    r = S.spar_sink_ot(a, b, x, y, eps=eps, s=s, tol=tol, max_iter=max_iter, dtype="f32", kdtype=kdtype,
                       seed=seed, cost_norm=S.COST_SCALE, cost_scale=cm, log_domain=1, sampler=sampler)
    inst = S.mlp_instance(x, a, y, b, cm, eps)
    al, be = r["alpha"].clone(), r["beta"].clone()
    S.mlp_gauge_fix(inst, al, be)
    return inst, al, be, r


def train(net: WarmStart, data, steps, lr=1e-3, lr_end=1e-4, log=None):
    """Adam over the training instances (one instance per step, cycling), with
    a cosine learning-rate decay from lr to lr_end."""
    losses = []
    for k in range(steps):
        inst, al, be = data[k % len(data)]
        c = 0.5 * (1.0 + math.cos(math.pi * k / max(1, steps - 1)))
        losses.append(net.train_step(inst, al, be, lr_end + (lr - lr_end) * c))
        if log and (k % 200 == 0 or k == steps - 1):
            log(f"step {k}: loss {losses[-1]:.4g}")
    return losses
