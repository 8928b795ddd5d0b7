"""Pins of the comparison rule the classifier parity tests use
(`oracle_pipeline.admissible`), on the CPU.

The learned classifier's label is the class of the largest logit when its
softmax probability reaches the threshold, else the exact CNA label.  The
parity tests accept, per row, any label that this rule can give when every
logit moves by up to the row's tolerance.  Checked here:
- with no tolerance exactly one label is admissible, the rule's own;
- admissible sets only grow with the tolerance;
- brute force: logits moved anywhere within the tolerance (random moves and
  the corners of the box) never give a label outside the admissible set.
"""
import numpy as np

import oracle_pipeline as op
from oracle import mlp as omlp


def _rule(logits, cna, threshold):
    p = omlp.softmax(logits)
    return np.where(p.max(1) >= threshold, p.argmax(1), cna)


def _rows(rng, n):
    scale = rng.choice([0.5, 2.0, 6.0, 15.0], n)
    logits = rng.normal(0.0, 1.0, (n, 4)) * scale[:, None]
    cna = rng.integers(0, 4, n)
    return logits, cna


def test_no_tolerance_admits_the_rule_alone():
    rng = np.random.default_rng(0)
    logits, cna = _rows(rng, 20000)
    for threshold in (0.5, 0.9, 0.99):
        ok, ambiguous = op.admissible(logits, np.zeros(len(logits)), cna, threshold)
        lab = _rule(logits, cna, threshold)
        # the softmax's single-precision allowance (1e-6) may admit the CNA
        # label as well on rows within 1e-6 of the threshold
        near = np.abs(omlp.softmax(logits).max(1) - threshold) < 2e-6
        assert ok[np.arange(len(lab)), lab].all()
        assert (ok.sum(1)[~near] == 1).all() and not ambiguous[~near].any()


def test_admissible_sets_grow_with_the_tolerance():
    rng = np.random.default_rng(1)
    logits, cna = _rows(rng, 20000)
    sets = [op.admissible(logits, np.full(len(logits), t), cna, 0.9)[0] for t in (0.0, 1e-3, 1e-2, 0.1, 0.5, 2.0)]
    for small, large in zip(sets, sets[1:]):
        assert (large | ~small).all()  # admissible at the smaller tolerance: admissible at the larger
    assert sets[-1].sum() > 1.2 * sets[0].sum()


def test_every_label_within_the_tolerance_is_admissible():
    rng = np.random.default_rng(2)
    n = 4000
    logits, cna = _rows(rng, n)
    tol = rng.choice([1e-3, 1e-2, 0.05, 0.2], n) * rng.uniform(0.5, 1.0, n)
    threshold = 0.9
    ok, _ = op.admissible(logits, tol, cna, threshold)
    # random moves inside the box |dl| <= tol, and its 16 corners
    corners = np.array(np.meshgrid(*[[-1.0, 1.0]] * 4, indexing="ij")).reshape(4, -1).T
    moves = [rng.uniform(-1.0, 1.0, (n, 4)) for _ in range(64)] + [np.broadcast_to(c, (n, 4)) for c in corners]
    for u in moves:
        lab = _rule(logits + u * tol[:, None], cna, threshold)
        assert ok[np.arange(n), lab].all()


def test_hand_worked_rows():
    """Threshold 0.9: logits (5, 0, 0, 0) give p = e^5 / (e^5 + 3) = 0.980 ->
    class 0; (2, 0, 0, 0) give p = 0.711 -> the CNA label, also with the
    leading two logits 0.001 apart and tolerance 0.01 (p = 0.48).
    Threshold 0.4: (3, 2.999, 0, 0) with tolerance 0.01 keep p = 0.48 above
    it, and either leading class may come out on top; (0.8, 0, 0, 0) give
    p = 0.426, which moves by at most 0.007 at tolerance 0.01 (the top class
    alone) and by up to 0.073 at tolerance 0.1 (the top class or, below the
    threshold, the CNA label)."""
    cna = np.array([3, 3, 3])
    logits = np.array([[5.0, 0, 0, 0], [2.0, 0, 0, 0], [3.0, 2.999, 0, 0]])
    ok, amb = op.admissible(logits, np.array([0.0, 0.0, 0.01]), cna, 0.9)
    assert ok.tolist() == [[True, False, False, False], [False, False, False, True], [False, False, False, True]]
    assert not amb.any()
    ok, amb = op.admissible(logits[2:], np.array([0.01]), cna[2:], 0.4)
    assert ok[0].tolist() == [True, True, False, False] and amb[0]
    row = np.array([[0.8, 0, 0, 0]])
    ok, amb = op.admissible(row, np.array([0.01]), cna[:1], 0.4)
    assert ok[0].tolist() == [True, False, False, False] and not amb[0]
    ok, amb = op.admissible(row, np.array([0.1]), cna[:1], 0.4)
    assert ok[0].tolist() == [True, False, False, True] and amb[0]
