"""mlp_oracle.py -- plain FP64 reference of the warm-start network.

TEST INFRASTRUCTURE ONLY: used by the tests to check the CUDA forward,
backward and Adam kernels.  It shares no code with the CUDA library.

The network (one per side; the source side predicts alpha, the target side
beta) follows its documented definition:
    f_i = [x_i / sqrt(cost_max), n a_i]                       (F = d + 1 features)
    P   = sum_j b_j relu(We g_j + ce) / sum_j b_j,  g_j = [y_j / sqrt(cost_max), m b_j]
    h1  = relu(W1 [f_i, P] + b1),  h2 = relu(W2 h1 + b2),  out_i = w3 . h2 + b3
and the training loss per side is
    L = sum_i a_i [target_i finite] ((out_i - target_i) / eps)^2 / sum_i a_i [target_i finite].
Gradients are written out by the chain rule (textbook backpropagation) and
pinned by the tests against central finite differences.  Adam follows Kingma &
Ba (2015), Algorithm 1, with bias correction.
"""
import numpy as np

E = 16
H = 128


def layout(d):
    """Offsets of one side's parameters (the documented order)."""
    F = d + 1
    D0 = F + E
    o = {}
    k = 0
    for name, size in (("We", E * F), ("ce", E), ("W1", H * D0), ("b1", H), ("W2", H * H), ("b2", H),
                       ("w3", H), ("b3", 1)):
        o[name] = (k, size)
        k += size
    o["size"] = k
    o["F"], o["D0"] = F, D0
    return o


def count(d):
    return 2 * layout(d)["size"]


def _unpack(w, d):
    o = layout(d)
    F, D0 = o["F"], o["D0"]
    g = lambda nm: w[o[nm][0]:o[nm][0] + o[nm][1]]
    return {"We": g("We").reshape(E, F), "ce": g("ce"), "W1": g("W1").reshape(H, D0), "b1": g("b1"),
            "W2": g("W2").reshape(H, H), "b2": g("b2"), "w3": g("w3"), "b3": g("b3")[0]}


def _relu(z):
    return np.maximum(z, 0.0)


def side_forward(w_side, d, sp, sw, op, ow, cost_max):
    """Prediction of one side and the intermediate values for backprop."""
    p = _unpack(np.asarray(w_side, np.float64), d)
    s = 1.0 / np.sqrt(cost_max)
    f = np.concatenate([np.asarray(sp, np.float64) * s, (len(sw) * np.asarray(sw, np.float64))[:, None]], 1)
    g = np.concatenate([np.asarray(op, np.float64) * s, (len(ow) * np.asarray(ow, np.float64))[:, None]], 1)
    ze = g @ p["We"].T + p["ce"]
    e = _relu(ze)
    wo = np.asarray(ow, np.float64)
    P = (wo @ e) / wo.sum()
    h0 = np.concatenate([f, np.repeat(P[None, :], len(sw), 0)], 1)
    z1 = h0 @ p["W1"].T + p["b1"]
    h1 = _relu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = _relu(z2)
    out = h2 @ p["w3"] + p["b3"]
    cache = dict(p=p, f=f, g=g, ze=ze, wo=wo, h0=h0, z1=z1, h1=h1, z2=z2, h2=h2)
    return out, cache


def side_loss_grad(w_side, d, sp, sw, op, ow, cost_max, target, eps):
    """Loss of one side and its gradient with respect to the side's parameters."""
    out, c = side_forward(w_side, d, sp, sw, op, ow, cost_max)
    p = c["p"]
    t = np.asarray(target, np.float64)
    fin = np.isfinite(t)
    a = np.where(fin, np.asarray(sw, np.float64), 0.0)
    W = a.sum()
    r = np.where(fin, out - np.where(fin, t, 0.0), 0.0)
    loss = float((a * r * r).sum() / (W * eps * eps))
    dout = 2.0 * a * r / (W * eps * eps)                       # dL/dout_i
    g = {}
    g["w3"] = c["h2"].T @ dout
    g["b3"] = dout.sum()
    dz2 = np.outer(dout, p["w3"]) * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["h0"]
    g["b1"] = dz1.sum(0)
    F = d + 1
    dP = (dz1 @ p["W1"])[:, F:].sum(0)                          # P enters every row of h0
    dze = np.outer(c["wo"] / c["wo"].sum(), dP) * (c["ze"] > 0)
    g["We"] = dze.T @ c["g"]
    g["ce"] = dze.sum(0)
    o = layout(d)
    gv = np.zeros(o["size"])
    for nm in ("We", "ce", "W1", "b1", "W2", "b2", "w3"):
        gv[o[nm][0]:o[nm][0] + o[nm][1]] = np.asarray(g[nm]).ravel()
    gv[o["b3"][0]] = g["b3"]
    return loss, gv


def loss_grad(w, d, x, a, y, b, cost_max, alpha_t, beta_t, eps):
    """Both sides: total loss and gradient (source side first)."""
    n = layout(d)["size"]
    la, ga = side_loss_grad(w[:n], d, x, a, y, b, cost_max, alpha_t, eps)
    lb, gb = side_loss_grad(w[n:], d, y, b, x, a, cost_max, beta_t, eps)
    return la + lb, np.concatenate([ga, gb])


def predict(w, d, x, a, y, b, cost_max):
    n = layout(d)["size"]
    al, _ = side_forward(w[:n], d, x, a, y, b, cost_max)
    be, _ = side_forward(w[n:], d, y, b, x, a, cost_max)
    return al, be


def gauge_fix(a, alpha, b, beta):
    """(alpha + c, beta - c) with sum a alpha = sum b beta over finite entries."""
    fa, fb = np.isfinite(alpha), np.isfinite(beta)
    sa = (a[fa] * alpha[fa]).sum()
    sb = (b[fb] * beta[fb]).sum()
    c = (sb - sa) / (a[fa].sum() + b[fb].sum())
    return np.where(fa, alpha + c, alpha), np.where(fb, beta - c, beta)


def adam(w, m1, m2, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Kingma & Ba, Algorithm 1 (bias-corrected moments)."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** step)
    vh = m2 / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m1, m2
