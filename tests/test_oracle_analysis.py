"""Pins of the FP64 oracle's bond order analysis, common neighbour analysis,
classifier features and MLP reference (no GPU)."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import mlp
from synth import configs, make_lattice
from synth.configs import R_CNA, random_box

RHO = 0.8442
LATTICE_CELLS = {"fcc": 4, "hcp": (5, 3, 3), "bcc": 5}


def _perfect(kind):
    lat = make_lattice(kind, LATTICE_CELLS[kind], RHO)
    return lat.sites(), lat.box


@pytest.mark.parametrize("kind", ["fcc", "hcp", "bcc"])
def test_perfect_lattice_Q_matches_paper_table(kind, golden):
    pos, box = _perfect(kind)
    offs, nbr = oracle.neighbours_brute(pos, box, 1.5)
    ref = golden["Q_table"][kind]
    for l, key in ((4, "Q4"), (5, "Q5"), (6, "Q6")):
        Q, nnb = oracle.boa(pos, box, offs, nbr, 1.5, l)
        assert (nnb == (14 if kind == "bcc" else 12)).all()
        # the paper prints three digits
        assert np.abs(Q - ref[key]).max() <= 0.0006, (kind, l, Q[0])


def test_boa_tolerance_table_is_the_papers(golden):
    codes = {1: "fcc", 2: "hcp", 3: "bcc"}
    for code, q4, q6 in oracle.BOA_TABLE:
        ref = golden["Q_table"][codes[code]]
        assert (q4, q6) == (ref["Q4"], ref["Q6"])


@pytest.mark.parametrize("kind,code", [("fcc", 1), ("hcp", 2), ("bcc", 3)])
def test_boa_tolerance_labels_perfect_lattices(kind, code):
    """Sec. 4.1: Q_l of a perfect lattice (computed by the oracle from its
    positions) lies within the paper's three printed digits of the table,
    so a tight tolerance labels every atom with its own lattice and no
    other."""
    pos, box = _perfect(kind)
    offs, nbr = oracle.neighbours_brute(pos, box, 1.5)
    q4, _ = oracle.boa(pos, box, offs, nbr, 1.5, 4)
    q6, _ = oracle.boa(pos, box, offs, nbr, 1.5, 6)
    lab, d = oracle.boa_tolerance_labels(q4, q6, 0.002)
    assert (lab == code).all() and d.max() < 0.001
    # half the distance to the nearest other lattice's point still labels it;
    # a tolerance below the three-digit rounding leaves it "other"
    assert (oracle.boa_tolerance_labels(q4, q6, 0.04)[0] == code).all()
    assert (oracle.boa_tolerance_labels(q4, q6, 1e-6)[0] == 0).all()


def _exact_ties(a, b):
    """Points near the midpoint of table points a and b whose two distances,
    evaluated in double precision as the rule evaluates them, are equal bit
    for bit (the midpoint itself is not: its two distances differ in the
    last place)."""
    k = np.arange(-64, 65)
    m4, m6 = 0.5 * (a[0] + b[0]), 0.5 * (a[1] + b[1])
    q4, q6 = np.broadcast_arrays(m4 + k[:, None] * np.spacing(m4), m6 + k[None, :] * np.spacing(m6))
    da = np.sqrt((q4 - a[0]) ** 2 + (q6 - a[1]) ** 2)
    db = np.sqrt((q4 - b[0]) ** 2 + (q6 - b[1]) ** 2)
    tie = da == db
    return q4[tie], q6[tie]


def test_boa_tolerance_rule_edges():
    """Strict tolerance, nearest point wins, table order on an exact tie,
    far points are other."""
    fcc, hcp, bcc = (0.191, 0.575), (0.097, 0.485), (0.036, 0.511)
    # exact ties: the earlier lattice of the table wins
    for (a, code), b in (((fcc, 1), hcp), ((hcp, 2), bcc)):
        q4, q6 = _exact_ties(a, b)
        assert len(q4) > 0
        lab, _ = oracle.boa_tolerance_labels(q4, q6, 1.0)
        assert (lab == code).all()
    # the distance equal to the tolerance, bit for bit: q6 - 0.575 is exact
    # (the operands are within a factor two of each other), and the square
    # root of a rounded square gives back the number in binary64
    q6 = 0.575 + 0.05
    tol = q6 - 0.575
    lab, d = oracle.boa_tolerance_labels([0.191], [q6], tol)
    assert d[0] == tol and lab[0] == 0  # a distance equal to the tolerance is not within it
    assert oracle.boa_tolerance_labels([0.191], [q6], np.nextafter(tol, 1.0))[0][0] == 1
    lab, _ = oracle.boa_tolerance_labels([0.191], [0.575 + 0.0499], 0.05)
    assert lab[0] == 1
    lab, _ = oracle.boa_tolerance_labels([0.0, 0.5], [0.0, 0.1], 0.3)
    assert (lab == 0).all()
    lab, _ = oracle.boa_tolerance_labels([0.04, 0.1], [0.51, 0.49], 0.02)
    assert list(lab) == [3, 2]


@pytest.mark.parametrize("seed", [1, 2])
def test_Q_direct_equals_addition_theorem(seed):
    """Two independent routes to Q_l: sums of Y_l^m (Eq. (5)) and the Legendre
    addition theorem."""
    pos, box = random_box(150, [6.0, 6.0, 6.0], seed, cutoffs=(1.5,), margin=1e-6, min_dist=0.8)
    offs, nbr = oracle.neighbours_brute(pos, box, 1.5)
    for l in (2, 3, 4, 6, 8):
        Qd, nnb = oracle.boa(pos, box, offs, nbr, 1.5, l)
        Qa = oracle.boa(pos, box, offs, nbr, 1.5, l, method="addition")
        assert np.abs(Qd - Qa).max() < 1e-12
        assert (Qd[nnb == 0] == 0).all()
    # l = 0: Y_0^0 is constant, so Q_0 = 1 for every atom with a neighbour
    Q0, nnb = oracle.boa(pos, box, offs, nbr, 1.5, 0)
    assert np.allclose(Q0[nnb > 0], 1.0, atol=1e-14)


def _rotation(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def test_Q_rotation_and_translation_invariant():
    rng = np.random.default_rng(3)
    cluster = rng.normal(0, 0.7, (40, 3))
    cluster = cluster[np.linalg.norm(cluster, axis=1) < 2.0]
    box = np.array([40.0, 40.0, 40.0])
    base = cluster + 20.0
    offs, nbr = oracle.neighbours_brute(base, box, 1.5)
    Q6a, _ = oracle.boa(base, box, offs, nbr, 1.5, 6)
    rot = cluster @ _rotation(4).T + np.array([13.3, 21.7, 19.1])
    Q6b, _ = oracle.boa(rot, box, offs, nbr, 1.5, 6)
    assert np.abs(Q6a - Q6b).max() < 1e-12


def _sig(nbond, trip, i):
    out = {}
    for t in trip[i, :nbond[i]]:
        k = f"{t >> 16},{(t >> 8) & 255},{t & 255}"
        out[k] = out.get(k, 0) + 1
    return out


@pytest.mark.parametrize("kind", ["fcc", "hcp", "bcc"])
def test_perfect_lattice_cna_signatures(kind, golden):
    pos, box = _perfect(kind)
    offs, nbr = oracle.neighbours_brute(pos, box, R_CNA)
    nbond, trip, partner, numax = oracle.cna(pos, box, offs, nbr, R_CNA)
    ref = golden["cna_signatures"][kind]
    for i in range(len(pos)):
        assert nbond[i] == ref["nbonds"]
        assert _sig(nbond, trip, i) == ref["triplets"]
    lab = oracle.cna_label(nbond, trip)
    assert (lab == {"fcc": 1, "hcp": 2, "bcc": 3}[kind]).all()


def _cna_brute(pos, box, rc):
    """Independent CNA: adjacency sets, common neighbours by intersection,
    largest component by union-find, counted in edges."""
    n = len(pos)
    dr = pos[:, None, :] - pos[None, :, :]
    dr -= box * np.rint(dr / box)
    adj = ((dr ** 2).sum(-1) < rc * rc) & ~np.eye(n, dtype=bool)
    nb = [set(np.nonzero(adj[i])[0].tolist()) for i in range(n)]
    out = {}
    for i in range(n):
        for j in nb[i]:
            C = nb[i] & nb[j]
            E = [(v, w) for v, w in itertools.combinations(sorted(C), 2) if w in nb[v]]
            parent = {v: v for v in C}

            def find(x):
                while parent[x] != x:
                    parent[x] = parent[parent[x]]
                    x = parent[x]
                return x
            for v, w in E:
                parent[find(v)] = find(w)
            count = {}
            for v, w in E:
                r = find(v)
                count[r] = count.get(r, 0) + 1
            out[(i, j)] = (len(C), len(E), max(count.values()) if count else 0)
    return out


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_cna_matches_brute_force(seed):
    pos, box = random_box(100, [5.2, 5.0, 4.9], seed, cutoffs=(R_CNA,), margin=1e-6, min_dist=0.8)
    offs, nbr = oracle.neighbours_brute(pos, box, 2.0)
    nbond, trip, partner, numax = oracle.cna(pos, box, offs, nbr, R_CNA)
    ref = _cna_brute(pos, box, R_CNA)
    seen = set()
    for i in range(len(pos)):
        for a in range(nbond[i]):
            j = int(partner[i, a])
            t = trip[i, a]
            assert (int(t >> 16), int((t >> 8) & 255), int(t & 255)) == ref[(i, j)]
            seen.add((i, j))
    assert seen == set(ref)
    # the triplet of a bond does not depend on which end computes it
    tmap = {(i, int(partner[i, a])): trip[i, a] for i in range(len(pos)) for a in range(nbond[i])}
    assert all(tmap[(j, i)] == t for (i, j), t in tmap.items())
    # the random boxes exercise split common-neighbour graphs (n_lcb < n_b)
    assert len(set(ref.values())) >= 5 and any(v[2] < v[1] for v in ref.values())


def test_cna_label_rule_needs_the_exact_signature():
    """Sec. 4.2's signatures, exactly: fcc 12 bonds all (4,2,1); hcp 12 bonds,
    six (4,2,1) and six (4,2,2); bcc 14 bonds, eight (6,6,6) and six
    (4,4,4).  Any other count or mix is other."""
    t421, t422 = oracle.triplet(4, 2, 1), oracle.triplet(4, 2, 2)
    t444, t666, t311 = oracle.triplet(4, 4, 4), oracle.triplet(6, 6, 6), oracle.triplet(3, 1, 1)
    rows = [
        (12, [t421] * 12, 1), (12, [t421] * 6 + [t422] * 6, 2), (14, [t666] * 8 + [t444] * 6, 3),
        (12, [t421] * 11 + [t311], 0), (12, [t421] * 10 + [t422] * 2, 0), (12, [t421] * 7 + [t422] * 5, 0),
        (12, [t421] * 5 + [t422] * 7, 0), (12, [t422] * 12, 0), (13, [t421] * 13, 0), (11, [t421] * 11, 0),
        (14, [t666] * 7 + [t444] * 7, 0), (14, [t666] * 9 + [t444] * 5, 0), (13, [t666] * 8 + [t444] * 5, 0),
        (15, [t666] * 8 + [t444] * 7, 0), (14, [t421] * 14, 0), (0, [], 0),
    ]
    mb = 16
    nbond = np.array([r[0] for r in rows], np.int32)
    trip = np.full((len(rows), mb), 0xFFFFFFFF, np.uint32)
    for k, (nb, ts, _) in enumerate(rows):
        trip[k, :len(ts)] = ts
    assert oracle.cna_label(nbond, trip).tolist() == [r[2] for r in rows]


def test_bond_order_of_an_atom_without_bonds_is_zero():
    """Atoms 3 apart have no neighbour within the bond-order cutoff: nu = 0
    and, by the convention of Eqs. (4)-(5), Q_l = 0 for every l."""
    k = np.arange(4)
    pos = 3.0 * np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    box = np.full(3, 12.0)
    offs, nbr = oracle.neighbours_brute(pos, box, 3.5)
    assert (np.diff(offs) > 0).all()  # listed neighbours, none of them bonded
    for l in (4, 5, 6):
        Q, nnb = oracle.boa(pos, box, offs, nbr, 1.5, l)
        assert (nnb == 0).all() and (Q == 0).all()
        assert (oracle.boa(pos, box, offs, nbr, 1.5, l, method="addition") == 0).all()


def test_cna_labels_permutation_invariant():
    c = configs.structure_box("hcp", 0.05, seed=9, cells=(6, 3, 3))
    pos, box = c["pos"], c["box"]
    perm = np.random.default_rng(1).permutation(len(pos))
    offs, nbr = oracle.neighbours_brute(pos, box, R_CNA)
    lab = oracle.cna_label(*oracle.cna(pos, box, offs, nbr, R_CNA)[:2])
    o2, n2 = oracle.neighbours_brute(pos[perm], box, R_CNA)
    lab2 = oracle.cna_label(*oracle.cna(pos[perm], box, o2, n2, R_CNA)[:2])
    assert np.array_equal(lab[perm], lab2)
    assert (lab == 2).sum() > 0


def _tent14(values, lo, width):
    """Reference tent histogram (14 bins of `width` centred on lo + width (b + 1/2))."""
    h = np.zeros(14)
    for v in values:
        x = (v - lo) / width - 0.5
        b0 = int(np.floor(x))
        t = x - b0
        if b0 < 0:
            h[0] += 1
        elif b0 >= 13:
            h[13] += 1
        else:
            h[b0] += 1 - t
            h[b0 + 1] += t
    return h


def test_features_perfect_fcc_closed_form():
    pos, box = _perfect("fcc")
    offs, nbr = oracle.neighbours_brute(pos, box, 1.5)
    f = oracle.features(pos, box, offs, nbr, 1.5, R_CNA)
    d = (4.0 / RHO) ** (1.0 / 3.0) / np.sqrt(2.0)
    expect = np.zeros(30)
    expect[0], expect[1] = 0.19094065395649334, 0.5745242597140697
    expect[2:14] = (d - R_CNA) / (1.5 - R_CNA)
    expect[14:16] = 1.0
    # 66 pairs of the 12 bonded neighbours: chords d (60 deg, 24 pairs),
    # sqrt2 d (90, 12), sqrt3 d (120, 24), 2 d (180, 6)
    chords = [d] * 24 + [np.sqrt(2) * d] * 12 + [np.sqrt(3) * d] * 24 + [2 * d] * 6
    expect[16:] = _tent14(chords, R_CNA - 0.35, 0.05) / 24.0
    assert np.abs(f - expect).max() < 1e-9


def test_features_shell_between_the_cutoffs():
    """fcc stretched so that its first shell (12 neighbours at d) lies between
    the bond length r_ref and the feature cutoff 1.5: Q4 and Q6 (taken over
    every neighbour within 1.5) are fcc's, the 12 distances are listed and
    the two missing ones are 1, and no pair is bonded, so the chord
    histogram is empty.  Q over the bonded neighbours only, or bonds taken
    at the feature cutoff, change these values."""
    d = 1.46
    assert R_CNA < d < 1.5
    a = d * np.sqrt(2.0)
    lat = make_lattice("fcc", (4, 4, 4), 4.0 / a ** 3)
    pos = lat.sites()
    offs, nbr = oracle.neighbours_brute(pos, lat.box, 1.5)
    f = oracle.features(pos, lat.box, offs, nbr, 1.5, R_CNA)
    expect = np.zeros(30)
    expect[0], expect[1] = 0.19094065395649334, 0.5745242597140697
    expect[2:14] = (d - R_CNA) / (1.5 - R_CNA)
    expect[14:16] = 1.0
    assert np.abs(f - expect).max() < 1e-9


def test_features_rotation_invariant_and_counts():
    rng = np.random.default_rng(8)
    cluster = rng.normal(0, 0.6, (30, 3))
    box = np.array([40.0, 40.0, 40.0])
    a = cluster + 20.0
    b = cluster @ _rotation(9).T + 17.5
    offs, nbr = oracle.neighbours_brute(a, box, 1.5)
    fa = oracle.features(a, box, offs, nbr, 1.5, R_CNA)
    fb = oracle.features(b, box, offs, nbr, 1.5, R_CNA)
    assert np.abs(fa - fb).max() < 1e-9
    # the chord histogram holds one unit per pair of bonded neighbours
    dist = np.sqrt(((a[:, None] - a[None]) ** 2).sum(-1))
    np.fill_diagonal(dist, np.inf)
    nb = (dist < R_CNA).sum(1)
    assert np.allclose(fa[:, 16:].sum(1) * 24.0, nb * (nb - 1) / 2)
    assert (np.diff(fa[:, 2:16], axis=1) >= -1e-15).all()


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(rng)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(0, 0.1, p[k].shape)
    x = rng.normal(0, 1, (16, 30))
    y = rng.integers(0, 4, 16)
    p = mlp.fit_input_norm(p, rng.normal(0.2, 0.5, (64, 30)))
    loss, g = mlp.loss_and_grad(p, x, y)
    h = 1e-6
    for k in p:
        if k in ("mu", "isd"):
            assert (g[k] == 0).all()  # fitted, not trained
            continue
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss_and_grad(p, x, y)[0]
            flat[idx] = old - h
            lm = mlp.loss_and_grad(p, x, y)[0]
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(fd)), k


def test_mlp_input_standardisation():
    """fit_input_norm gives the standardised training features zero mean and
    unit variance (a constant feature passes through unscaled), and the
    forward pass with (mu, isd) equals the unstandardised network applied to
    (x - mu) isd."""
    rng = np.random.default_rng(3)
    x = rng.normal(rng.uniform(-2, 2, 30), rng.uniform(0.1, 3.0, 30), (500, 30))
    x[:, 4] = 0.7
    p = mlp.fit_input_norm(mlp.init_params(rng), x)
    z = (x - p["mu"]) * p["isd"]
    keep = np.arange(30) != 4
    assert np.allclose(z.mean(0), 0.0, atol=1e-12)
    assert np.allclose(z[:, keep].std(0), 1.0, rtol=1e-12)
    assert p["isd"][4] == 1.0 and np.abs(z[:, 4]).max() < 1e-12
    q = dict(p, mu=np.zeros(30), isd=np.ones(30))
    assert np.allclose(mlp.forward(p, x)[0], mlp.forward(q, z)[0], rtol=1e-12, atol=1e-12)
    # AdamW leaves the standardisation alone
    g = {k: np.ones_like(v) for k, v in p.items()}
    mu0, isd0 = p["mu"].copy(), p["isd"].copy()
    mlp.adamw_step(p, g, mlp.adamw_init(p), lr=0.1, wd=0.5)
    assert np.array_equal(p["mu"], mu0) and np.array_equal(p["isd"], isd0)


def test_softmax_of_large_logits():
    """Softmax is unchanged by a common shift of the logits, and stays finite
    for logits far beyond exp's range (the largest logit is taken out
    first)."""
    rng = np.random.default_rng(4)
    z = rng.normal(0, 3, (100, 4))
    assert np.allclose(mlp.softmax(z), mlp.softmax(z + 700.0), rtol=1e-12, atol=0)
    p = mlp.softmax(np.array([[1000.0, 0.0, -1000.0, 999.0]]))
    assert np.isfinite(p).all() and abs(p.sum() - 1.0) < 1e-15
    assert np.allclose(p, [[1 / (1 + np.exp(-1.0)), 0.0, 0.0, np.exp(-1.0) / (1 + np.exp(-1.0))]], rtol=1e-14)


def test_adamw_textbook_steps():
    """Three parameters, two steps, against values worked out by hand from the
    AdamW update (bias-corrected moments, decoupled decay on weights)."""
    p = {"W1": np.array([1.0, -2.0, 0.5])}
    s = mlp.adamw_init(p)
    g1 = {"W1": np.array([0.1, 0.0, -0.4])}
    mlp.adamw_step(p, g1, s, lr=0.1, wd=0.5, eps=1e-8)
    # step 1: m_hat = g, v_hat = g^2 -> update g/(|g| + eps) = sign(g) (or 0)
    exp1 = np.array([1.0 * (1 - 0.05) - 0.1 * (0.1 / (0.1 + 1e-8)),
                     -2.0 * (1 - 0.05),
                     0.5 * (1 - 0.05) + 0.1 * (0.4 / (0.4 + 1e-8))])
    assert np.allclose(p["W1"], exp1, rtol=0, atol=1e-12)
    g2 = {"W1": np.array([0.3, 0.2, 0.0])}
    mlp.adamw_step(p, g2, s, lr=0.1, wd=0.5, eps=1e-8)
    m = 0.9 * 0.1 * np.array([0.1, 0.0, -0.4]) + 0.1 * np.array([0.3, 0.2, 0.0])
    v = 0.999 * 0.001 * np.array([0.01, 0.0, 0.16]) + 0.001 * np.array([0.09, 0.04, 0.0])
    mh, vh = m / (1 - 0.81), v / (1 - 0.999 ** 2)
    exp2 = exp1 * (1 - 0.05) - 0.1 * mh / (np.sqrt(vh) + 1e-8)
    assert np.allclose(p["W1"], exp2, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------
# Adaptive CNA
# ---------------------------------------------------------------------------
ACNA_F = (1.0 + np.sqrt(2.0)) / 2.0
ACNA_CELLS = {"fcc": (4, 4, 4), "hcp": (5, 3, 3), "bcc": (5, 5, 5)}


@pytest.mark.parametrize("kind,code", [("fcc", 1), ("hcp", 2), ("bcc", 3)])
@pytest.mark.parametrize("scale", [0.8, 1.0, 1.3])
def test_acna_perfect_lattices_at_any_density(kind, code, scale):
    """The point of the adaptive cutoff: perfect lattices are recognised at
    any density (a fixed-cutoff CNA at 1.433625 would not be), and the local
    cutoff is f d_nn (fcc, hcp) or f a (bcc) in closed form."""
    rho = 0.8442 / scale ** 3
    lat = make_lattice(kind, ACNA_CELLS[kind], rho)
    pos, box = lat.sites(), lat.box
    offs, nb = oracle.neighbours_cells(pos, box, 1.8 * scale)
    lab, rc = oracle.acna(pos, box, offs, nb)
    assert (lab == code).all()
    if kind == "bcc":
        a = (2.0 / rho) ** (1.0 / 3.0)
        assert np.allclose(rc[:, 1], ACNA_F * a, rtol=1e-12)
    else:
        d_nn = (np.sqrt(2.0) / rho) ** (1.0 / 3.0)
        assert np.allclose(rc[:, 0], ACNA_F * d_nn, rtol=1e-12)
        assert (rc[:, 1] == 0).all()


def test_acna_scale_invariance_is_exact():
    """Doubling every length (a power of two: every FP64 operation scales
    exactly) leaves every label unchanged and doubles every cutoff."""
    pos, box = _mixed_box(seed=5)
    offs, nb = oracle.neighbours_cells(pos, box, 1.8)
    lab, rc = oracle.acna(pos, box, offs, nb)
    offs2, nb2 = oracle.neighbours_cells(2.0 * pos, 2.0 * box, 3.6)
    lab2, rc2 = oracle.acna(2.0 * pos, 2.0 * box, offs2, nb2)
    assert np.array_equal(lab, lab2)
    assert np.array_equal(2.0 * rc, rc2)
    assert len(set(lab.tolist())) >= 2  # the box mixes ordered and disordered environments


def _mixed_box(seed):
    """A small noisy box: fcc, bcc or hcp environments and disordered ones."""
    rng = np.random.default_rng(seed)
    lat = make_lattice("fcc", (5, 5, 5), 0.8442)
    pos = lat.sites() + rng.normal(0.0, 0.06, (len(lat.sites()), 3))
    # a disordered slab
    sl = pos[:, 2] < lat.box[2] * 0.3
    pos[sl] += rng.normal(0.0, 0.25, (sl.sum(), 3))
    return pos - lat.box * np.floor(pos / lat.box), np.asarray(lat.box, float)


def _acna_numpy(pos, box, offs, nb):
    """Adaptive CNA written independently: dense adjacency matrices and
    scipy's connected components for the largest cluster."""
    from scipy.sparse.csgraph import connected_components
    f, c = (1.0 + np.sqrt(2.0)) * 0.5, 2.0 / np.sqrt(3.0)
    n = len(pos)
    out = np.zeros(n, np.int8)

    def r2(a, b):
        t = pos[a] - pos[b]
        t = t - box * np.rint(t / box)
        return t[..., 0] * t[..., 0] + t[..., 1] * t[..., 1] + t[..., 2] * t[..., 2]

    def signatures(sel, rc):
        rc2 = rc * rc
        A = r2(sel[:, None], sel[None, :]) < rc2
        np.fill_diagonal(A, False)
        sig = []
        for a in range(len(sel)):
            cn = np.flatnonzero(A[a])
            sub = A[np.ix_(cn, cn)]
            ne = int(sub.sum()) // 2
            best = 0
            if ne:
                k, comp = connected_components(sub.astype(np.int8), directed=False)
                for q in range(k):
                    m = comp == q
                    best = max(best, int(sub[np.ix_(m, m)].sum()) // 2)
            sig.append((len(cn), ne, best))
        return sig

    for i in range(n):
        js = nb[offs[i]:offs[i + 1]]
        d2 = r2(np.full(len(js), i), js)
        order = np.lexsort((js, d2))
        js, d2 = js[order], d2[order]
        lab = 0
        if len(js) >= 12:
            s = 0.0
            for v in d2[:12]:
                s += np.sqrt(v)
            sig = signatures(js[:12], f * (s / 12.0))
            if sig.count((4, 2, 1)) == 12:
                lab = 1
            elif sig.count((4, 2, 1)) == 6 and sig.count((4, 2, 2)) == 6:
                lab = 2
        if lab == 0 and len(js) >= 14:
            s8 = s6 = 0.0
            for k, v in enumerate(d2[:14]):
                if k < 8:
                    s8 += np.sqrt(v)
                else:
                    s6 += np.sqrt(v)
            sig = signatures(js[:14], f * ((c * s8 + s6) / 14.0))
            if sig.count((6, 6, 6)) == 8 and sig.count((4, 4, 4)) == 6:
                lab = 3
        out[i] = lab
    return out


@pytest.mark.parametrize("kind", ["fcc", "bcc", "hcp", "mixed"])
def test_acna_matches_independent_numpy_version(kind):
    if kind == "mixed":
        pos, box = _mixed_box(seed=9)
    else:
        c = configs.structure_box(kind, 0.07, 8, cells={"fcc": (4, 4, 4), "bcc": (5, 5, 5), "hcp": (5, 3, 3)}[kind])
        pos, box = c["pos"], np.asarray(c["box"], float)
    offs, nb = oracle.neighbours_cells(pos, box, 1.8)
    lab, _ = oracle.acna(pos, box, offs, nb)
    assert np.array_equal(lab, _acna_numpy(pos, box, offs, nb))
    assert (lab > 0).any()
