"""FP64 reference of the learned structure classifier (NumPy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network: inputs standardised x' = (x - mu) isd (mu, isd fitted to the
training features, not trained), then 30 -> 64 -> 64 -> 4, ReLU after the
two hidden layers, softmax output over the classes (0 other, 1 fcc, 2 hcp,
3 bcc).  Loss: mean cross
entropy over the batch.  Optimiser: AdamW (Loshchilov & Hutter, decoupled
weight decay) with beta = (0.9, 0.999), eps = 1e-8; the decay applies to the
weight matrices only.  Initialisation: He-uniform weights
U(-sqrt(6/fan_in), sqrt(6/fan_in)), zero biases.

Weight layout: W1[30, 64], W2[64, 64], W3[64, 4] (input-major, y = x @ W + b).
"""
from __future__ import annotations

import numpy as np

SIZES = (30, 64, 64, 4)
NAMES = ("mu", "isd", "W1", "b1", "W2", "b2", "W3", "b3")


def init_params(rng: np.random.Generator):
    p = {"mu": np.zeros(SIZES[0]), "isd": np.ones(SIZES[0])}
    for k in range(3):
        fi, fo = SIZES[k], SIZES[k + 1]
        lim = np.sqrt(6.0 / fi)
        p[f"W{k + 1}"] = rng.uniform(-lim, lim, size=(fi, fo))
        p[f"b{k + 1}"] = np.zeros(fo)
    return p


def fit_input_norm(p, x):
    """mu, isd = mean and 1/standard deviation of every input feature."""
    p["mu"] = x.mean(axis=0)
    var = x.var(axis=0)
    p["isd"] = np.where(var > 1e-12, 1.0 / np.sqrt(np.maximum(var, 1e-300)), 1.0)
    return p


def forward(p, x):
    """Returns (logits, cache); the cache holds the standardised inputs."""
    x = (x - p["mu"]) * p["isd"]
    z1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    logits = h2 @ p["W3"] + p["b3"]
    return logits, (x, z1, h1, z2, h2)


def bf16_round(a):
    """Nearest BF16 value (round to nearest, ties to even) of each FP32
    value of `a`, returned as float64.  BF16 keeps the sign, the 8 exponent
    bits and the top 7 fraction bits of an IEEE single; the dropped 16 bits
    round the kept part."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + keep_lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, x):
    """The network with BF16 operands, as the classifier is specified (BF16
    weights and activations, wider accumulation): the standardisation in
    single precision, (x - mu) then * isd, each rounded to FP32; the
    standardised inputs and both hidden activations rounded to BF16 before
    they enter the next layer; the weight matrices rounded to BF16; biases
    in FP32; every sum of products accumulated in FP64.  x: BF16 values
    (float64 array).  Returns (logits, (xs, z1, h1, z2, h2))."""
    f32 = lambda v: np.asarray(v, dtype=np.float32)
    W1, W2, W3 = (bf16_round(p[k]) for k in ("W1", "W2", "W3"))
    xs = bf16_round((f32(x) - f32(p["mu"])) * f32(p["isd"]))
    z1 = xs @ W1 + f32(p["b1"]).astype(np.float64)
    h1 = bf16_round(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + f32(p["b2"]).astype(np.float64)
    h2 = bf16_round(np.maximum(z2, 0.0))
    logits = h2 @ W3 + f32(p["b3"]).astype(np.float64)
    return logits, (xs, z1, h1, z2, h2)


def softmax(logits):
    z = logits - logits.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def loss_and_grad(p, x, y):
    """Mean cross entropy and its gradient with respect to every parameter."""
    logits, (x, z1, h1, z2, h2) = forward(p, x)
    prob = softmax(logits)
    n = len(x)
    loss = -np.mean(np.log(prob[np.arange(n), y]))
    g3 = prob.copy()
    g3[np.arange(n), y] -= 1.0
    g3 /= n
    grads = {"W3": h2.T @ g3, "b3": g3.sum(0)}
    d2 = (g3 @ p["W3"].T) * (z2 > 0)
    grads["W2"] = h1.T @ d2
    grads["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"].T) * (z1 > 0)
    grads["W1"] = x.T @ d1
    grads["b1"] = d1.sum(0)
    grads["mu"] = np.zeros_like(p["mu"])  # standardisation is not trained
    grads["isd"] = np.zeros_like(p["isd"])
    return loss, grads


def adamw_init(p):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()}, "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adamw_step(p, grads, state, lr=1e-3, wd=0.01, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW update in place: m, v moments, bias correction, decoupled decay."""
    state["t"] += 1
    t = state["t"]
    for k in p:
        if k in ("mu", "isd"):
            continue  # fitted, not trained
        g = grads[k]
        m = state["m"][k] = b1 * state["m"][k] + (1.0 - b1) * g
        v = state["v"][k] = b2 * state["v"][k] + (1.0 - b2) * g * g
        mh = m / (1.0 - b1 ** t)
        vh = v / (1.0 - b2 ** t)
        if k.startswith("W"):
            p[k] = p[k] - lr * wd * p[k]
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
