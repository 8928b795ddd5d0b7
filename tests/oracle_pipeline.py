"""Oracle-side classifier pipeline for the parity tests (test infrastructure).

Everything here is computed by the FP64 oracle from seeded synthetic inputs;
nothing comes from the CUDA library:
  - a trained-scale parameter vector: the oracle's network trained with the
    oracle's AdamW on oracle features labelled by the oracle's CNA;
  - per box: oracle features rounded to BF16 (as the library stores them),
    the oracle's BF16-operand network (`oracle.mlp.forward_bf16`), and the
    oracle's exact CNA labels;
  - per row, the logit tolerance of that comparison (`flip_tolerance`).

Tolerance.  The library and `forward_bf16` round the same operands to BF16
at the same points; they differ in the accumulation (FP32 on the tensor
cores, FP64 in the oracle), which moves a sum by at most ~K 2^-24 of its
absolute terms, and, through it, in the rare activation that lands on the
other side of a BF16 rounding boundary: one BF16 step (2^-7 of the value's
leading power of two) of one activation, whose effect on each logit is that
step times the row's Jacobian entry (the network is piecewise linear).  A
row's tolerance is the accumulation term plus the largest single-step effect
in each layer (hidden layers always; the input layer only where the two
sides' inputs may differ, i.e. features computed on both sides, and then
doubled, since one input step moves every hidden unit).  Checked on the CPU
against an FP32-accumulating emulation (tests/test_oracle_mlp_bf16.py).
The functions are module-level so that a `spawn` process pool can run them.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import mlp as omlp
from synth import configs
from synth.configs import R_BOA, R_CNA

BLOCKS = [("mu", 0, 30, (30,)), ("isd", 30, 60, (30,)), ("W1", 60, 1980, (30, 64)), ("b1", 1980, 2044, (64,)),
          ("W2", 2044, 6140, (64, 64)), ("b2", 6140, 6204, (64,)), ("W3", 6204, 6460, (64, 4)),
          ("b3", 6460, 6464, (4,))]
ACC_REL = 1e-4  # FP32 accumulation of <= 64 products, with margin


def pack(p):
    return np.concatenate([p[name].reshape(-1) for name, *_ in BLOCKS])


def unpack(v):
    return {name: np.asarray(v[a:b], dtype=np.float64).reshape(shape) for name, a, b, shape in BLOCKS}


def bf16_step(v):
    """One BF16 rounding step at |v| (2^-7 of its leading power of two; 0 at 0)."""
    a = np.abs(v)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 0.0)


def structure_rows(seed, kinds=("fcc", "bcc", "hcp", "liquid"), sigmas=(0.02, 0.06, 0.1), cells=None):
    """Oracle features (FP64) and oracle CNA labels of small structure boxes."""
    cells = cells or {"fcc": (10, 10, 5), "bcc": (10, 10, 5), "hcp": (10, 6, 6), "liquid": (12, 12, 12)}
    xs, ys = [], []
    for kind in kinds:
        for s in sigmas:
            c = configs.structure_box(kind, s, seed, cells=cells[kind])
            xs.append(features_of(c["pos"], c["box"]))
            ys.append(cna_labels_of(c["pos"], c["box"]))
    return np.concatenate(xs), np.concatenate(ys)


def features_of(pos, box):
    offs, nb = oracle.neighbours_cells(pos, box, R_BOA)
    return oracle.features(pos, box, offs, nb, R_BOA, R_CNA)


def cna_labels_of(pos, box):
    offs, nb = oracle.neighbours_cells(pos, box, R_CNA)
    return oracle.cna_label(*oracle.cna(pos, box, offs, nb, R_CNA)[:2])


def train_params(seed=61, steps=600, batch=4096, lr=3e-3):
    """A trained-scale network: the oracle's AdamW on oracle features
    (BF16-rounded, standardised to the training rows) and CNA labels.
    Returned as the library holds it: one FP32 vector."""
    x, y = structure_rows(seed)
    x = omlp.bf16_round(x)
    rng = np.random.default_rng(seed)
    p = omlp.fit_input_norm(omlp.init_params(rng), x)
    st = omlp.adamw_init(p)
    for _ in range(steps):
        idx = rng.integers(0, len(x), batch)
        _, g = omlp.loss_and_grad(p, x[idx], y[idx])
        omlp.adamw_step(p, g, st, lr=lr, wd=0.01)
    return pack(p).astype(np.float32)


def flip_tolerance(q, x, fwd, inputs_differ):
    """Per row (see the module docstring): ACC_REL of the absolute logit
    sums plus, per layer, the largest |Jacobian| x one BF16 step."""
    xs, z1, h1, z2, h2 = fwd
    W1, W2, W3 = (omlp.bf16_round(q[k]) for k in ("W1", "W2", "W3"))
    # units within accumulation error of zero count as live (a flip can turn them on)
    m1 = (z1 > -ACC_REL * np.abs(z1).max(1, keepdims=True)).astype(np.float64)
    m2 = (z2 > -ACC_REL * np.abs(z2).max(1, keepdims=True)).astype(np.float64)
    K2 = m2[:, :, None] * W3[None]  # d logits / d h2  [n, 64, 4]
    K1 = np.stack([K2[:, :, c] @ W2.T for c in range(4)], axis=2)  # d logits / d h1 (before its mask)
    tol = ACC_REL * (np.abs(h2) @ np.abs(W3) + np.abs(q["b3"])).max(1)
    tol += (bf16_step(h2)[:, :, None] * np.abs(K2)).max(axis=(1, 2))
    tol += (bf16_step(h1)[:, :, None] * np.abs(K1)).max(axis=(1, 2))
    # the hidden layers' own accumulation errors end in their BF16 rounding
    # (no change, or one of the steps above); the standardised inputs are the
    # same bits on both sides when the BF16 inputs are
    if inputs_differ:
        J0 = np.stack([(m1 * K1[:, :, c]) @ W1.T for c in range(4)], axis=2)  # d logits / d xs
        # one BF16 step of a feature, standardised, and of its rounded image
        step = bf16_step(x) * np.abs(q["isd"]) + bf16_step(xs)
        tol += (step[:, :, None] * np.abs(J0)).max(axis=(1, 2))
        # an input step moves every hidden unit, and more than one of them
        # may then round the other way: twice the single-step budget
        tol *= 2.0
    return tol


def admissible(logits, tol, cna, threshold):
    """Labels the pipeline may return for each row when every logit may move
    by up to tol: the classes whose logit can reach the top if the largest
    softmax probability can stay >= threshold, and the CNA label if it can
    fall below it.  Returns a [n, 4] boolean mask of classes and a flag of
    rows with more than one admissible label."""
    n = len(logits)
    top = logits.max(1)
    cand = logits >= (top - 2.0 * tol)[:, None]
    # largest softmax probability range over the perturbation
    pr = omlp.softmax(logits)
    pmax = pr.max(1)
    # first order |dp| <= 2 p (1 - p) max|dl|; 1.5x for the second order,
    # 1e-6 for the library's single-precision softmax
    dp = 3.0 * pmax * (1.0 - pmax) * tol + 1e-6
    can_keep = pmax + dp >= threshold
    can_fall = pmax - dp < threshold
    ok = np.zeros((n, 4), dtype=bool)
    ok[can_keep] = cand[can_keep]
    rows = np.nonzero(can_fall)[0]
    ok[rows, cna[rows]] = True
    return ok, ok.sum(1) > 1


def classify_box(args):
    """One box through the oracle pipeline: oracle features (BF16), the
    oracle's BF16-operand network, the tolerance of each row (with input
    flips: the library computes its features in single precision), and the
    exact CNA labels.  Returns (logits, tol, cna)."""
    pos, box, pv = args
    q = unpack(pv)
    xb = omlp.bf16_round(features_of(pos, box))
    logits, fwd = omlp.forward_bf16(q, xb)
    tol = flip_tolerance(q, xb, fwd, inputs_differ=True)
    return logits, tol, cna_labels_of(pos, box)


def classifier_box_through_oracle(args):
    """Box k of the classifier inference set built in this process
    (synth.configs.classifier_box), then classify_box.  Returns (pos, box,
    logits, tol, cna)."""
    seed, k, pv = args
    b = configs.classifier_box(seed, k)
    logits, tol, cna = classify_box((b["pos"], b["box"], pv))
    return b["pos"], b["box"], logits, tol, cna
