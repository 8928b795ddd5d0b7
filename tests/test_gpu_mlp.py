"""GPU parity of the learned classifier: features, tensor-core MLP forward,
gradients, AdamW, training and the classification pipeline, against the
FP64 oracle.

Tolerances: features |d| <= 2e-5 (single precision; Q_l as in BOA);
logits |d| <= 0.03 max(1, rms logit) (BF16 inputs, weights and activations,
FP32 accumulation: 2^-9 relative per rounding through three layers);
weight gradients per block: norm error <= 2^-7 (four BF16 roundings of
2^-9) times the norm of the same block computed from absolute values
(|A|^T |D|, the running error bound of a sum of products whose operands are
rounded), and cosine >= 0.999, against the oracle evaluated on the same
BF16-rounded inputs and weights;
AdamW in FP32 against FP64: <= 1e-5 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle_pipeline as op
from oracle import mlp as omlp
from synth import configs
from synth.configs import R_BOA, R_CNA

pytestmark = pytest.mark.gpu
BLOCKS = [("mu", 0, 30, (30,)), ("isd", 30, 60, (30,)), ("W1", 60, 1980, (30, 64)), ("b1", 1980, 2044, (64,)),
          ("W2", 2044, 6140, (64, 64)), ("b2", 6140, 6204, (64,)), ("W3", 6204, 6460, (64, 4)),
          ("b3", 6460, 6464, (4,))]


@pytest.fixture(scope="module")
def L():
    from paper_1704_03329_b300 import lib
    return lib


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


def cu(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


def pack(p):
    return np.concatenate([p[name].reshape(-1) for name, *_ in BLOCKS])


def unpack(v):
    return {name: v[a:b].reshape(shape) for name, a, b, shape in BLOCKS}


def _params(seed, bias_scale=0.1, standardise=True):
    """Random parameters; with standardise, a non-trivial mu and isd (the
    inputs below are drawn around 0.3 with spread 0.4)."""
    rng = np.random.default_rng(seed)
    p = omlp.init_params(rng)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(0, bias_scale, p[k].shape)
    if standardise:
        p["mu"] = rng.uniform(0.1, 0.5, 30)
        p["isd"] = rng.uniform(1.0, 4.0, 30)
    return p


def _box(kind, sigma, seed=33):
    cells = {"fcc": (10, 10, 5), "bcc": (10, 10, 5), "hcp": (10, 6, 6), "liquid": (12, 12, 12)}[kind]
    return configs.structure_box(kind, sigma, seed, cells=cells)


@pytest.mark.parametrize("kind", ["fcc", "bcc", "hcp", "liquid"])
def test_features_parity(L, ctx, kind):
    c = _box(kind, 0.05)
    pos, box = c["pos"], c["box"]
    offs, nb = oracle.neighbours_cells(pos, box, R_BOA)
    fo = oracle.features(pos, box, offs, nb, R_BOA, R_CNA)
    f, fb = L.ppmd_features(ctx, cu(pos), box, R_BOA, fp32=True, bf16=True, r_ref=R_CNA)
    f = f.cpu().numpy()
    assert np.abs(f - fo).max() <= 2e-5
    fb = fb.to(torch.float32).cpu().numpy()
    assert np.abs(fb[:, :30] - f).max() <= 2 ** -8 * max(1.0, np.abs(f).max())
    assert (fb[:, 30:] == 0).all()


def test_mlp_forward_parity(L, ctx):
    p = _params(1)
    rng = np.random.default_rng(2)
    x = rng.normal(0.3, 0.4, (1000, 30))
    xb = np.zeros((1000, 32))
    xb[:, :30] = x
    x_bf = bf16_round(xb)
    pq = {k: bf16_round(v) if k.startswith("W") else v for k, v in p.items()}
    ref, _ = omlp.forward(pq, x_bf[:, :30])
    logits = L.ppmd_mlp_forward(ctx, cu(pack(p), torch.float32), cu(x_bf, torch.bfloat16)).cpu().numpy()
    scale = max(1.0, np.sqrt((ref ** 2).mean()))
    assert np.abs(logits - ref).max() <= 0.03 * scale
    agree = (logits.argmax(1) == ref.argmax(1)).mean()
    assert agree >= 0.99


def _abs_grad_scale(p, x, y):
    """Per block, the norm of the gradient evaluated with every product
    replaced by the product of absolute values."""
    logits, (xs, z1, h1, z2, h2) = omlp.forward(p, x)
    g3 = omlp.softmax(logits)
    g3[np.arange(len(x)), y] -= 1.0
    g3 = np.abs(g3) / len(x)
    d2 = (g3 @ np.abs(p["W3"]).T) * (z2 > 0)
    d1 = (d2 @ np.abs(p["W2"]).T) * (z1 > 0)
    blocks = {"W3": np.abs(h2).T @ g3, "b3": g3.sum(0), "W2": np.abs(h1).T @ d2, "b2": d2.sum(0),
              "W1": np.abs(xs).T @ d1, "b1": d1.sum(0)}
    return {k: np.linalg.norm(v) for k, v in blocks.items()}


def _cos(a, b):
    return float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


@pytest.mark.parametrize("batch", [4096, 1000])
def test_mlp_gradients_parity(L, ctx, batch):
    p = _params(3)
    rng = np.random.default_rng(4)
    xb = np.zeros((batch, 32))
    xb[:, :30] = rng.normal(0.3, 0.4, (batch, 30))
    y = rng.integers(0, 4, batch)
    x_bf = bf16_round(xb)
    pq = {k: bf16_round(v) if k.startswith("W") else v for k, v in p.items()}
    loss_o, g_o = omlp.loss_and_grad(pq, x_bf[:, :30], y)
    grad, loss = L.ppmd_mlp_grad(ctx, cu(pack(p), torch.float32), cu(x_bf, torch.bfloat16), cu(y, torch.int8))
    g = unpack(grad.cpu().numpy().astype(np.float64))
    scale = _abs_grad_scale(pq, x_bf[:, :30], y)
    assert abs(float(loss.cpu()) - loss_o) <= 1e-3 * loss_o
    for name, *_ in BLOCKS:
        a, b = g[name].reshape(-1), g_o[name].reshape(-1)
        if name in ("mu", "isd"):
            assert (a == 0).all(), name  # the standardisation is not trained
            continue
        assert np.linalg.norm(a - b) <= 2 ** -7 * scale[name], name
        assert _cos(a, b) >= 0.999, name


def test_adamw_matches_oracle(L, ctx):
    p = _params(5)
    rng = np.random.default_rng(6)
    pv = pack(p)
    P = cu(pv, torch.float32)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    state = omlp.adamw_init(p)
    for step in (1, 2, 3):
        gv = rng.normal(0, 0.05, pv.shape)
        L.ppmd_mlp_adamw(ctx, P, M, V, cu(gv, torch.float32), step, lr=1e-3, wd=0.01)
        omlp.adamw_step(p, unpack(gv), state, lr=1e-3, wd=0.01)
    got = P.cpu().numpy().astype(np.float64)
    ref = pack(p)
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.array_equal(got[:60], pv[:60].astype(np.float32))  # mu, isd untouched


def test_fit_input_norm(L, ctx):
    rng = np.random.default_rng(9)
    n = 5000
    xb = np.zeros((n, 32))
    xb[:, :30] = rng.normal(rng.uniform(-1, 1, 30), rng.uniform(0.05, 2.0, 30), (n, 30))
    xb[:, 7] = 0.25  # a constant feature keeps isd = 1
    x_bf = bf16_round(xb)
    p = _params(10, standardise=False)
    P = cu(pack(p), torch.float32)
    L.ppmd_mlp_fit_input_norm(ctx, P, cu(x_bf, torch.bfloat16))
    q = omlp.fit_input_norm(dict(p), x_bf[:, :30])
    got = P.cpu().numpy().astype(np.float64)
    assert np.allclose(got[:30], q["mu"], rtol=1e-6, atol=1e-6)
    assert np.allclose(got[30:60], q["isd"], rtol=1e-4)
    assert got[30 + 7] == 1.0
    assert np.array_equal(got[60:], pack(p)[60:].astype(np.float32))


def _training_set(L, ctx, seed):
    xs, ys = [], []
    for kind in ("fcc", "bcc", "hcp", "liquid"):
        for sigma in (0.02, 0.06, 0.1):
            c = _box(kind, sigma, seed)
            p = cu(c["pos"])
            _, fb = L.ppmd_features(ctx, p, c["box"], R_BOA, fp32=False, bf16=True)
            lab, _, _ = L.ppmd_classify(ctx, p, c["box"], mode=0, r_cna=R_CNA)
            xs.append(fb)
            ys.append(lab)
    return torch.cat(xs), torch.cat(ys)


def test_training_learns_cna_labels(L, ctx):
    """A few hundred AdamW steps on CNA-labelled structure boxes: the loss
    falls and held-out atoms are classified like CNA."""
    x, y = _training_set(L, ctx, 41)
    xt, yt = _training_set(L, ctx, 42)
    rng = np.random.default_rng(7)
    P = cu(pack(omlp.init_params(rng)), torch.float32)
    L.ppmd_mlp_fit_input_norm(ctx, P, x)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cpu").manual_seed(0)
    losses = []
    B = 4096
    for step in range(1, 401):
        idx = torch.randint(0, x.shape[0], (B,), generator=g).cuda()
        L.ppmd_mlp_train_step(ctx, P, M, V, step, x[idx].contiguous(), y[idx].contiguous(), lr=3e-3, wd=0.01, loss=loss)
        if step % 50 == 0:
            losses.append(float(loss.cpu()))
    assert losses[-1] < 0.5 * losses[0]
    logits = L.ppmd_mlp_forward(ctx, P, xt)
    agree = (logits.argmax(1).to(torch.int8) == yt).float().mean().item()
    assert agree >= 0.9, agree
    # with the CNA fallback below confidence 0.9 the labels follow CNA closely
    c = _box("hcp", 0.06, 43)
    pc = cu(c["pos"])
    exact, _, _ = L.ppmd_classify(ctx, pc, c["box"], mode=0, r_cna=R_CNA)
    lab, conf, nfb = L.ppmd_classify(ctx, pc, c["box"], mode=1, params=P, threshold=0.9)
    lab0, _, _ = L.ppmd_classify(ctx, pc, c["box"], mode=1, params=P, threshold=0.0)
    both = (lab == exact).float().mean().item()
    alone = (lab0 == exact).float().mean().item()
    # the fallback only replaces low-confidence labels with the exact ones, so
    # on the same box it can only raise the agreement
    low = conf < 0.9
    assert torch.equal(lab[low], exact[low]) and torch.equal(lab[~low], lab0[~low])
    assert both >= 0.95 and both >= alone, (both, alone, nfb / len(c["pos"]))


def test_classify_modes(L, ctx):
    c = _box("fcc", 0.06, 44)
    p = cu(c["pos"])
    exact, _, nfb0 = L.ppmd_classify(ctx, p, c["box"], mode=0, r_cna=R_CNA)
    offs, nb = oracle.neighbours_cells(c["pos"], c["box"], R_BOA)
    lab_o = oracle.cna_label(*oracle.cna(c["pos"], c["box"], offs, nb, R_CNA)[:2])
    assert np.array_equal(exact.cpu().numpy(), lab_o)
    params = cu(pack(_params(8)), torch.float32)
    # threshold above 1: every atom falls back to CNA
    lab, conf, nfb = L.ppmd_classify(ctx, p, c["box"], mode=1, params=params, threshold=1.01)
    assert nfb == len(c["pos"]) and np.array_equal(lab.cpu().numpy(), lab_o)
    # threshold 0: no fallback, labels are the MLP's argmax over the features
    lab, conf, nfb = L.ppmd_classify(ctx, p, c["box"], mode=1, params=params, threshold=0.0)
    assert nfb == 0
    _, fb = L.ppmd_features(ctx, p, c["box"], R_BOA, fp32=False, bf16=True)
    logits = L.ppmd_mlp_forward(ctx, params, fb)
    assert torch.equal(lab, logits.argmax(1).to(torch.int8))
    pr = torch.softmax(logits, 1).max(1).values
    assert torch.allclose(conf, pr, atol=1e-5)


@pytest.fixture(scope="module")
def trained_vec():
    """Trained-scale parameters made by the oracle alone (oracle features,
    CNA labels, AdamW in FP64), as the library's FP32 vector."""
    return op.train_params()


def test_mlp_forward_every_tile_pass_trained(L, ctx, trained_vec):
    """The tensor-core forward pass in its steady state: the grid is at most
    148 x 4 CTAs, each taking two 128-row tiles per pass of its two-slot
    loop, so 500,037 rows give every CTA at least three passes (mbarrier
    phases cycled, both slots refilled, tensor memory reused) and a ragged
    last tile.  Rows: oracle features of the four structures at three noise
    levels, and rows drawn around them.  Every logit is compared with the
    oracle's BF16-operand network within the row's flip tolerance, and with
    the FP64-activation network at the forward test's tolerance; the argmax
    must match wherever the top two logits are further apart than twice the
    row's tolerance."""
    n = 500037
    assert n >= 2 * 148 * 4 * 128 * 3
    cells = {"fcc": (20, 20, 10), "bcc": (20, 20, 20), "hcp": (20, 12, 12), "liquid": (24, 24, 24)}
    xs, _ = op.structure_rows(63, cells=cells)
    rng = np.random.default_rng(64)
    extra = rng.normal(xs.mean(0), xs.std(0) + 1e-3, (n - len(xs), 30))
    x = omlp.bf16_round(np.concatenate([xs, extra]))
    x = x[rng.permutation(n)]
    xb = np.zeros((n, 32))
    xb[:, :30] = x
    q = op.unpack(trained_vec.astype(np.float64))
    logits = L.ppmd_mlp_forward(ctx, cu(trained_vec, torch.float32), cu(xb, torch.bfloat16)).cpu().numpy()
    ref, fwd = omlp.forward_bf16(q, x)
    tol = op.flip_tolerance(q, x, fwd, inputs_differ=False)
    err = np.abs(logits - ref).max(1)
    assert (err <= tol).all(), (float((err / tol).max()), int(np.argmax(err / tol)))
    # the FP64-activation network at the forward test's tolerance
    qb = dict(q, W1=omlp.bf16_round(q["W1"]), W2=omlp.bf16_round(q["W2"]), W3=omlp.bf16_round(q["W3"]))
    ref64 = omlp.forward(qb, x)[0]
    assert np.abs(logits - ref64).max() <= 0.03 * max(1.0, np.sqrt((ref64 ** 2).mean()))
    srt = np.sort(ref, 1)
    clear = srt[:, -1] - srt[:, -2] > 2.0 * tol
    assert clear.mean() > 0.99
    assert np.array_equal(logits.argmax(1)[clear], ref.argmax(1)[clear])
