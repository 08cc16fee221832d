"""CPU oracle of the learned region surrogate (TEST INFRASTRUCTURE ONLY).

Plain PyTorch CPU operations in float64, written from the surrogate's
definition: features, a D -> H -> H -> 1 MLP with the tanh form of GELU
(Hendrycks & Gimpel 2016), weights rounded to bfloat16, activations rounded to
bfloat16 after each GELU (`round_act`), and the region output transform. The
gradient of the mean squared error comes from torch autograd on the same
function without activation rounding (the rounding's derivative is taken as
the identity), so it can be pinned by finite differences. Adam follows Kingma
& Ba (2014). Parameter layout: W1 [H][D], b1 [H], W2 [H][H], b2 [H], W3 [H], b3.
"""
from __future__ import annotations

import math

import numpy as np
import torch

GELU_A = math.sqrt(2.0 / math.pi)
GELU_B = 0.044715


def bf16(t):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    return t.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def gelu(z):
    return 0.5 * z * (1.0 + torch.tanh(GELU_A * (z + GELU_B * z ** 3)))


def unpack(p, D, H):
    p = torch.as_tensor(np.asarray(p, dtype=np.float64))
    o = 0
    W1 = p[o:o + H * D].reshape(H, D); o += H * D
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o:o + 1]; o += 1
    return [W1, b1, W2, b2, W3, b3]


def n_params(D, H):
    return H * D + H + H * H + H + H + 1


def features(kind, x, param):
    """(n, D) float64 features and the output multiplier of each invocation.
    Black-Scholes: ln(S/K), sigma sqrt T, r T, d1 clamped to [-10, 10], sigma."""
    x = torch.as_tensor(np.asarray(x, dtype=np.float64))
    if kind == 0:      # Black-Scholes: S, K, T, sigma
        S, K, T, sig = x[0], x[1], x[2], x[3]
        d1 = (torch.log(S / K) + (param + 0.5 * sig * sig) * T) / (sig * torch.sqrt(T))
        f = torch.stack([torch.log(S / K), sig * torch.sqrt(T), param * T,
                         torch.clamp(d1, -10.0, 10.0), sig], dim=1)
        return f, S
    # EOS (e, v1, dv, q): the multiplier is the ideal-gas pressure of the energy
    # after the viscous work, (gamma - 1) max(e - dv q, 0) / v1
    e, v1, dv, q = x[0], x[1], x[2], x[3]
    mult = (param - 1.0) * torch.clamp(e - dv * q, min=0.0) / v1
    return x[:4].T.clone(), mult


def net(params, desc, f, round_act=True):
    """Network output for normalised features f (n, D); weights rounded to bf16."""
    D, H = desc["n_feat"], desc["hidden"]
    W1, b1, W2, b2, W3, b3 = params
    fn = (f - torch.tensor(desc["feat_shift"][:D], dtype=torch.float64)) * \
        torch.tensor(desc["feat_scale"][:D], dtype=torch.float64)
    z1 = fn @ bf16(W1).T + b1
    h1 = gelu(z1)
    if round_act:
        h1 = bf16(h1)
    z2 = h1 @ bf16(W2).T + b2
    h2 = gelu(z2)
    if round_act:
        h2 = bf16(h2)
    return h2 @ bf16(W3) + b3, (fn, z1, h1, z2, h2)


def forward(p, desc, kind, x, param, round_act=True):
    """Region outputs of the surrogate (n,) and the network outputs."""
    params = unpack(p, desc["n_feat"], desc["hidden"])
    f, mult = features(kind, x, param)
    y, inter = net(params, desc, f, round_act)
    out = mult * (desc["out_shift"] + desc["out_scale"] * y)
    if kind == 1:
        out = torch.clamp(out, min=0.0)   # pressure is non-negative
    return out.numpy(), y.numpy(), inter


def loss_and_grad(p, desc, kind, x, param, target):
    """Mean squared error of the network against normalised targets and its
    gradient with respect to the parameters (bf16-rounded weights as leaves)."""
    D, H = desc["n_feat"], desc["hidden"]
    leaves = [t.clone().requires_grad_(True) for t in unpack(p, D, H)]
    f, mult = features(kind, x, param)
    t = torch.as_tensor(np.asarray(target, dtype=np.float64))
    used = mult != 0          # rows with a zero multiplier carry no target
    tn = torch.where(used, (t / torch.where(used, mult, 1.0) - desc["out_shift"]) / desc["out_scale"], 0.0)

    def fwd(ls):
        W1, b1, W2, b2, W3, b3 = ls
        fn = (f - torch.tensor(desc["feat_shift"][:D], dtype=torch.float64)) * \
            torch.tensor(desc["feat_scale"][:D], dtype=torch.float64)
        # weights enter through their bf16 values; the rounding passes gradients through
        w1 = W1 + (bf16(W1) - W1).detach()
        w2 = W2 + (bf16(W2) - W2).detach()
        w3 = W3 + (bf16(W3) - W3).detach()
        h1 = gelu(fn @ w1.T + b1)
        h2 = gelu(h1 @ w2.T + b2)
        return h2 @ w3 + b3

    y = fwd(leaves)
    loss = torch.mean(torch.where(used, y - tn, 0.0) ** 2)
    loss.backward()
    g = torch.cat([l.grad.reshape(-1) for l in leaves]).numpy()
    return float(loss.item()), g, fwd, leaves, tn


def input_grad(p, desc, kind, x, param):
    """d(region output)/d(region inputs) of the unrounded network, (4, n)."""
    D, H = desc["n_feat"], desc["hidden"]
    params = [bf16(t) if i in (0, 2, 4) else t for i, t in enumerate(unpack(p, D, H))]
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64)).clone().requires_grad_(True)
    if kind == 0:
        S, K, T, sig = xt[0], xt[1], xt[2], xt[3]
        d1 = (torch.log(S / K) + (param + 0.5 * sig * sig) * T) / (sig * torch.sqrt(T))
        f = torch.stack([torch.log(S / K), sig * torch.sqrt(T), param * T,
                         torch.clamp(d1, -10.0, 10.0), sig], dim=1)
        mult = S
    else:
        f = xt[:4].T
        e, v1, dv, q = xt[0], xt[1], xt[2], xt[3]
        mult = (param - 1.0) * torch.clamp(e - dv * q, min=0.0) / v1
    y, _ = net(params, desc, f, round_act=False)
    out = mult * (desc["out_shift"] + desc["out_scale"] * y)
    out.sum().backward()
    return xt.grad.numpy()


def vjp(p, desc, kind, x, param, gout):
    """Vector-Jacobian products of the region output (the EOS output clamped at
    zero, as served) of the unrounded network with bf16 weights: the gradient
    of sum_i gout_i out_i with respect to the parameters (the weights' bf16
    rounding passed through as the identity, as in loss_and_grad) and to the
    region inputs (4, n)."""
    D, H = desc["n_feat"], desc["hidden"]
    leaves = [t.clone().requires_grad_(True) for t in unpack(p, D, H)]
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64)).clone().requires_grad_(True)
    if kind == 0:
        S, K, T, sig = xt[0], xt[1], xt[2], xt[3]
        d1 = (torch.log(S / K) + (param + 0.5 * sig * sig) * T) / (sig * torch.sqrt(T))
        f = torch.stack([torch.log(S / K), sig * torch.sqrt(T), param * T,
                         torch.clamp(d1, -10.0, 10.0), sig], dim=1)
        mult = S
    else:
        f = xt[:4].T
        e, v1, dv, q = xt[0], xt[1], xt[2], xt[3]
        mult = (param - 1.0) * torch.clamp(e - dv * q, min=0.0) / v1
    W1, b1, W2, b2, W3, b3 = leaves
    fn = (f - torch.tensor(desc["feat_shift"][:D], dtype=torch.float64)) * \
        torch.tensor(desc["feat_scale"][:D], dtype=torch.float64)
    w1 = W1 + (bf16(W1) - W1).detach()
    w2 = W2 + (bf16(W2) - W2).detach()
    w3 = W3 + (bf16(W3) - W3).detach()
    y = gelu(gelu(fn @ w1.T + b1) @ w2.T + b2) @ w3 + b3
    out = mult * (desc["out_shift"] + desc["out_scale"] * y)
    if kind == 1:
        out = torch.clamp(out, min=0.0)
    g = torch.as_tensor(np.asarray(gout, dtype=np.float64))
    (out * g).sum().backward()
    return torch.cat([l.grad.reshape(-1) for l in leaves]).numpy(), xt.grad.numpy()


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2014) in float64; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def desc_dict(d):
    """Plain dict of an hpac_mlp_desc-like object (or dict)."""
    if isinstance(d, dict):
        return d
    return {"n_feat": d.n_feat, "hidden": d.hidden, "feat_shift": list(d.feat_shift),
            "feat_scale": list(d.feat_scale), "out_shift": d.out_shift, "out_scale": d.out_scale}
