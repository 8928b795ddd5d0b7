"""Pins of the oracle's BF16-operand network and of the logit tolerance the
classifier parity tests use (CPU only).

- bf16_round against PyTorch's float32 -> bfloat16 conversion (a library
  routine, round to nearest even), ties included;
- forward_bf16 equals the FP64 network exactly when every operand and every
  partial sum is representable in BF16 (small dyadic weights and inputs), so
  it computes the same network with nothing dropped or transposed; and it
  differs from it by rounding only on general inputs;
- the rounding points: every activation entering a product is a BF16 value
  (torch's conversion leaves it unchanged) and each hidden layer is its
  ReLU pre-activation rounded once; weights moved by less than a quarter
  BF16 step leave the logits unchanged;
- the tolerance: an emulation of the library's arithmetic (the same BF16
  rounding points, sums accumulated in FP32 instead of FP64) stays within
  flip_tolerance on every row of oracle features of the four structures,
  with identical inputs and with inputs one BF16 step apart.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
import oracle_pipeline as op


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(0, 3, 200000), rng.uniform(-1e-3, 1e-3, 20000)]).astype(np.float32)
    # exact ties: the dropped half is 0x8000 (round to the even neighbour)
    u = rng.integers(0, 2 ** 16, 5000).astype(np.uint32) << 16 | 0x8000
    ties = u.view(np.float32)
    ties = ties[np.isfinite(ties)]
    for v in (a, ties):
        ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(omlp.bf16_round(v), ref)


def _dyadic_params(rng):
    """Weights in {-1/2, 0, 1/2} with at most two non-zeros per output unit,
    biases multiples of 1/4 in [-1, 1], mu = 0, isd = 1: every activation of
    0/1 inputs is a multiple of 1/8 below 2^4, exact in BF16."""
    p = {"mu": np.zeros(30), "isd": np.ones(30)}
    for k, (fi, fo) in enumerate(((30, 64), (64, 64), (64, 4)), start=1):
        W = np.zeros((fi, fo))
        for j in range(fo):
            rows = rng.choice(fi, 2, replace=False)
            W[rows, j] = rng.choice([-0.5, 0.5], 2)
        p[f"W{k}"] = W
        p[f"b{k}"] = rng.integers(-4, 5, fo) / 4.0
    return p


def test_forward_bf16_is_the_network_on_exact_operands():
    rng = np.random.default_rng(1)
    p = _dyadic_params(rng)
    x = rng.integers(0, 2, (2000, 30)).astype(np.float64)
    a, (xs, z1, h1, z2, h2) = omlp.forward_bf16(p, x)
    b, cache = omlp.forward(p, x)
    assert np.array_equal(a, b)
    for u, v in zip((xs, z1, h1, z2, h2), cache):
        assert np.array_equal(u, v)
    assert (np.abs(h1) > 0).any() and (np.abs(h2) > 0).any()


def test_forward_bf16_differs_by_rounding_only():
    p = op.unpack(op.train_params().astype(np.float64))
    rng = np.random.default_rng(2)
    x = omlp.bf16_round(rng.normal(0.3, 0.4, (5000, 30)))
    a = omlp.forward_bf16(p, x)[0]
    b = omlp.forward(dict(p, W1=omlp.bf16_round(p["W1"]), W2=omlp.bf16_round(p["W2"]), W3=omlp.bf16_round(p["W3"])),
                     x)[0]
    d = np.abs(a - b)
    scale = np.sqrt((b ** 2).mean())
    assert 0 < d.max() <= 0.03 * scale  # three BF16 roundings of ~2^-9 each


def test_forward_bf16_operands_are_bf16_values():
    """Every activation that enters a product -- the standardised inputs and
    both hidden layers -- is a BF16 value (torch's FP32 -> BF16 conversion
    leaves it unchanged), and each hidden layer is its ReLU pre-activation
    rounded once: within half a BF16 step (2^-8 relative: eight significant
    bits) of it."""
    p = op.unpack(op.train_params().astype(np.float64))
    rng = np.random.default_rng(5)
    x = omlp.bf16_round(rng.normal(0.3, 0.4, (5000, 30)))
    _, (xs, z1, h1, z2, h2) = omlp.forward_bf16(p, x)

    def is_bf16(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
        return np.array_equal(t.to(torch.bfloat16).to(torch.float64).numpy(), a)

    for a in (xs, h1, h2):
        assert is_bf16(a)
    for z, h in ((z1, h1), (z2, h2)):
        r = np.maximum(z, 0.0)
        assert not is_bf16(r)  # the pre-activations are wider: the rounding is a real step
        assert np.all(np.abs(h - r) <= 2.0 ** -8 * r)
        assert (h > 0).any()


def test_forward_bf16_weights_enter_as_bf16():
    """The weight matrices enter as BF16 values: moving every weight by less
    than a quarter of its BF16 step (so that it rounds to the same BF16
    value) leaves the logits unchanged bit for bit."""
    p = op.unpack(op.train_params().astype(np.float64))
    rng = np.random.default_rng(6)
    x = omlp.bf16_round(rng.normal(0.3, 0.4, (2000, 30)))
    ref = omlp.forward_bf16(p, x)[0]
    for k in ("W1", "W2", "W3"):
        w = torch.from_numpy(p[k].astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
        step = op.bf16_step(w)
        moved = w + rng.uniform(-0.24, 0.24, w.shape) * step
        assert not np.array_equal(moved, w)
        q = dict(p, **{k: moved})
        assert np.array_equal(omlp.forward_bf16(q, x)[0], ref), k


def _emulate_fp32(q, x):
    """The library's arithmetic on the CPU: forward_bf16's rounding points,
    with every sum of products accumulated in FP32."""
    f32 = lambda v: np.asarray(v, dtype=np.float32)
    W1, W2, W3 = (f32(omlp.bf16_round(q[k])) for k in ("W1", "W2", "W3"))
    xs = omlp.bf16_round((f32(x) - f32(q["mu"])) * f32(q["isd"]))
    h1 = omlp.bf16_round(np.maximum(f32(f32(xs) @ W1) + f32(q["b1"]), 0))
    h2 = omlp.bf16_round(np.maximum(f32(f32(h1) @ W2) + f32(q["b2"]), 0))
    return (f32(f32(h2) @ W3) + f32(q["b3"])).astype(np.float64)


@pytest.fixture(scope="module")
def trained_and_rows():
    pv = op.train_params()
    x, _ = op.structure_rows(62)
    rng = np.random.default_rng(3)
    mu, sd = x.mean(0), x.std(0) + 1e-3
    x = np.concatenate([x, rng.normal(mu, sd, (20000, 30))])  # off-lattice rows with the same spread
    return op.unpack(pv.astype(np.float64)), omlp.bf16_round(x)


def test_tolerance_covers_fp32_accumulation(trained_and_rows):
    q, x = trained_and_rows
    ref, fwd = omlp.forward_bf16(q, x)
    tol = op.flip_tolerance(q, x, fwd, inputs_differ=False)
    d = np.abs(_emulate_fp32(q, x) - ref).max(1)
    assert (d > 0).mean() > 0.5  # the two accumulations really differ
    assert (d <= tol).all(), float((d / tol).max())


def test_tolerance_covers_one_feature_step(trained_and_rows):
    q, x = trained_and_rows
    rng = np.random.default_rng(4)
    # move one feature of each row by one BF16 step, as single-precision
    # features rounding on the other side of a boundary would
    k = rng.integers(0, 30, len(x))
    sgn = rng.choice([-1.0, 1.0], len(x))
    xp = x.copy()
    r = np.arange(len(x))
    xp[r, k] = omlp.bf16_round(x[r, k] + sgn * op.bf16_step(x[r, k]))
    ref, fwd = omlp.forward_bf16(q, x)
    tol = op.flip_tolerance(q, x, fwd, inputs_differ=True)
    d = np.abs(_emulate_fp32(q, xp) - ref).max(1)
    assert (d <= tol).all(), float((d / tol).max())
    # and the tolerance is useful: most rows keep a decision margin above it
    lg = np.sort(ref, 1)
    assert np.median(tol) < 0.1 * np.median(lg[:, -1] - lg[:, -2])
