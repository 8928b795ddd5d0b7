"""Several independent boxes in one analysis pipeline (ppmd_analyze_boxes,
ppmd_classify_boxes).

Each box's results equal the FP64 oracle's for that box alone: neighbour
counts and CNA labels bit for bit, Q4/Q6 within 1e-5 (single precision, as
for one box).  The learned classifier gives every atom the same label and
confidence as one call per box: the boxes keep their own cell grids, so
each atom sees the same list in the same order and the same arithmetic.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import configs
from synth.configs import R_BOA, R_CNA

pytestmark = pytest.mark.gpu
# five boxes of different structure, noise and size (different cell grids)
KINDS = [("fcc", 0.02, (10, 10, 5)), ("bcc", 0.1, (10, 10, 5)), ("hcp", 0.05, (10, 6, 6)),
         ("liquid", 0.0, (12, 12, 12)), ("fcc", 0.1, (7, 8, 9))]


@pytest.fixture(scope="module")
def L():
    from paper_1704_03329_b300 import lib
    return lib


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


def cu(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.fixture(scope="module")
def box_set():
    boxes = [configs.structure_box(k, s, 40 + i, cells=c) for i, (k, s, c) in enumerate(KINDS)]
    pos = np.concatenate([b["pos"] for b in boxes])
    off = np.cumsum([0] + [len(b["pos"]) for b in boxes]).tolist()
    return boxes, pos, off


def test_analyze_boxes_matches_oracle_per_box(L, ctx, box_set):
    boxes, pos, off = box_set
    out = L.ppmd_analyze_boxes(ctx, cu(pos), off, [b["box"] for b in boxes], R_BOA, R_CNA)
    ctx.sync()
    lab = out["label"].cpu().numpy()
    q4, q6, nnb = (out[k].cpu().numpy() for k in ("q4", "q6", "n_nb"))
    for b, lo, hi in zip(boxes, off[:-1], off[1:]):
        offs, nb = oracle.neighbours_cells(b["pos"], b["box"], R_BOA)
        Q4o, nno = oracle.boa(b["pos"], b["box"], offs, nb, R_BOA, 4)
        Q6o, _ = oracle.boa(b["pos"], b["box"], offs, nb, R_BOA, 6)
        lab_o = oracle.cna_label(*oracle.cna(b["pos"], b["box"], offs, nb, R_CNA)[:2])
        assert np.array_equal(lab[lo:hi], lab_o), b["kind"]
        assert np.array_equal(nnb[lo:hi], nno), b["kind"]
        assert np.abs(q4[lo:hi] - Q4o).max() <= 1e-5
        assert np.abs(q6[lo:hi] - Q6o).max() <= 1e-5


def test_analyze_boxes_one_box_is_analyze(L, ctx, box_set):
    boxes, _, _ = box_set
    b = boxes[2]
    p = cu(b["pos"])
    one = L.ppmd_analyze(ctx, p, b["box"], R_BOA, R_CNA)
    many = L.ppmd_analyze_boxes(ctx, p, [0, len(b["pos"])], [b["box"]], R_BOA, R_CNA)
    ctx.sync()
    for k in ("label", "q4", "q6", "n_nb"):
        assert torch.equal(one[k], many[k])


def _params(seed):
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(0.0, 0.6, 30), rng.uniform(0.5, 2.0, 30)]
    for fi, fo in ((30, 64), (64, 64), (64, 4)):
        lim = np.sqrt(6.0 / fi)
        parts += [rng.uniform(-lim, lim, fi * fo), rng.uniform(-0.1, 0.1, fo)]
    return np.concatenate(parts)


@pytest.mark.parametrize("threshold", [0.0, 0.6, 1.01])
def test_classify_boxes_equals_one_call_per_box(L, ctx, box_set, threshold):
    boxes, pos, off = box_set
    params = cu(_params(9), torch.float32)
    lab, conf, nfb = L.ppmd_classify_boxes(ctx, cu(pos), off, [b["box"] for b in boxes], mode=1, params=params,
                                           threshold=threshold)
    total = 0
    for b, lo, hi in zip(boxes, off[:-1], off[1:]):
        l1, c1, n1 = L.ppmd_classify(ctx, cu(b["pos"]), b["box"], mode=1, params=params, threshold=threshold)
        assert torch.equal(lab[lo:hi], l1), b["kind"]
        assert torch.equal(conf[lo:hi], c1), b["kind"]
        total += n1
    assert nfb == total
    if threshold > 1.0:  # every atom falls back: exact CNA of each box
        assert nfb == len(pos)
        exact, _, _ = L.ppmd_classify_boxes(ctx, cu(pos), off, [b["box"] for b in boxes], mode=0, r_cna=R_CNA)
        assert torch.equal(lab, exact)


def test_boxes_reject_bad_offsets(L, ctx, box_set):
    boxes, pos, off = box_set
    bad = list(off)
    bad[2], bad[3] = bad[3], bad[2]  # decreasing
    with pytest.raises(L.PPMDError) as ei:
        L.ppmd_analyze_boxes(ctx, cu(pos), bad, [b["box"] for b in boxes], R_BOA, R_CNA)
    assert ei.value.code == L.ERR_INVALID


def test_boxes_with_an_empty_box_and_all_empty(L, ctx, box_set):
    """An empty box in the middle of the set changes nothing for the others;
    a set of empty boxes gives empty outputs."""
    boxes, pos, off = box_set
    bx = [b["box"] for b in boxes]
    off2 = off[:3] + [off[2]] + off[3:]  # an empty box after the second
    bx2 = bx[:2] + [[9.0, 9.0, 9.0]] + bx[2:]
    ref = L.ppmd_analyze_boxes(ctx, cu(pos), off, bx, R_BOA, R_CNA)
    got = L.ppmd_analyze_boxes(ctx, cu(pos), off2, bx2, R_BOA, R_CNA)
    ctx.sync()
    for k in ("label", "q4", "q6", "n_nb"):
        assert torch.equal(ref[k], got[k])
    params = cu(_params(9), torch.float32)
    l1, c1, n1 = L.ppmd_classify_boxes(ctx, cu(pos), off, bx, mode=1, params=params, threshold=0.6)
    l2, c2, n2 = L.ppmd_classify_boxes(ctx, cu(pos), off2, bx2, mode=1, params=params, threshold=0.6)
    assert torch.equal(l1, l2) and torch.equal(c1, c2) and n1 == n2
    empty = cu(np.zeros((0, 3)))
    lab, conf, nfb = L.ppmd_classify_boxes(ctx, empty, [0, 0, 0], [[9.0, 9.0, 9.0], [8.0, 8.0, 8.0]], mode=1,
                                           params=params)
    out = L.ppmd_analyze_boxes(ctx, empty, [0, 0], [[9.0, 9.0, 9.0]], R_BOA, R_CNA)
    ctx.sync()
    assert lab.numel() == 0 and nfb == 0 and out["label"].numel() == 0


def test_classify_boxes_full_size_exact_mode(L, ctx):
    """The classifier suite's inference set at full size (32 boxes, 4,096,000
    atoms) through one box-set call in exact mode, as the bench times it:
    every label of four of the boxes against the oracle's CNA of that box."""
    test = configs.classifier_boxes(51)
    pos = np.concatenate([b["pos"] for b in test])
    off = np.cumsum([0] + [len(b["pos"]) for b in test]).tolist()
    assert off[-1] == 4096000
    lab, _, _ = L.ppmd_classify_boxes(ctx, cu(pos), off, [b["box"] for b in test], mode=0, r_cna=R_CNA)
    ctx.sync()
    lab = lab.cpu().numpy()
    for bi in (0, 9, 18, 27):
        b = test[bi]
        offs, nb = oracle.neighbours_cells(b["pos"], b["box"], R_CNA)
        lab_o = oracle.cna_label(*oracle.cna(b["pos"], b["box"], offs, nb, R_CNA)[:2])
        assert np.array_equal(lab[off[bi]:off[bi + 1]], lab_o), bi
