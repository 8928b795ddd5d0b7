"""GPU parity of bond order analysis (Q4, Q6) and common neighbour analysis
against the FP64 oracle.

Q_l are computed in single precision: |dQ| <= 1e-5 absolute.  Neighbour
counts, CNA triplets and structure labels are compared bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import configs, make_lattice
from synth.configs import R_BOA, R_CNA

pytestmark = pytest.mark.gpu
SMALL = {"fcc": (10, 10, 5), "bcc": (10, 10, 5), "hcp": (10, 6, 6), "liquid": (12, 12, 12)}


@pytest.fixture(scope="module")
def L():
    from paper_1704_03329_b300 import lib
    return lib


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


def cu(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _gpu_list(L, ctx, p, box, r, max_nbr=48):
    nc, cell_of, start, atoms = L.ppmd_build_cells(ctx, p, box, r)
    return L.ppmd_build_neighbours(ctx, p, box, r, start, atoms, nc, max_nbr)


def _box(kind, sigma, seed=31):
    return configs.structure_box(kind, sigma, seed, cells=SMALL[kind])


@pytest.mark.parametrize("kind", ["fcc", "bcc", "hcp", "liquid"])
@pytest.mark.parametrize("sigma", [0.02, 0.1])
def test_boa_parity(L, ctx, kind, sigma):
    c = _box(kind, sigma)
    pos, box = c["pos"], c["box"]
    offs, nb = oracle.neighbours_cells(pos, box, R_BOA)
    Q4o, nno = oracle.boa(pos, box, offs, nb, R_BOA, 4)
    Q6o, _ = oracle.boa(pos, box, offs, nb, R_BOA, 6)
    p = cu(pos)
    nbr, cnt = _gpu_list(L, ctx, p, box, R_BOA)
    q4, q6, nnb = L.ppmd_boa_q46(ctx, p, box, R_BOA, nbr, cnt)
    assert np.array_equal(nnb.cpu().numpy(), nno)
    assert np.abs(q4.cpu().numpy() - Q4o).max() <= 1e-5
    assert np.abs(q6.cpu().numpy() - Q6o).max() <= 1e-5


@pytest.mark.parametrize("kind", ["fcc", "bcc", "hcp"])
def test_boa_perfect_lattice_table(L, ctx, kind, golden):
    lat = make_lattice(kind, SMALL[kind], 0.8442)
    pos, box = lat.sites(), lat.box
    p = cu(pos)
    nbr, cnt = _gpu_list(L, ctx, p, box, R_BOA)
    q4, q6, nnb = L.ppmd_boa_q46(ctx, p, box, R_BOA, nbr, cnt)
    ref = golden["Q_table"][kind]
    assert np.abs(q4.cpu().numpy() - ref["Q4"]).max() <= 0.0006
    assert np.abs(q6.cpu().numpy() - ref["Q6"]).max() <= 0.0006


def _trip_map(nbr, cnt, trip):
    nbr, cnt, trip = nbr.cpu().numpy(), cnt.cpu().numpy(), trip.cpu().numpy().view(np.uint32)
    out = {}
    for i in range(len(cnt)):
        for m in range(cnt[i]):
            if trip[i, m] != 0xFFFFFFFF:
                out[(i, int(nbr[i, m]))] = int(trip[i, m])
    return out


@pytest.mark.parametrize("kind", ["fcc", "bcc", "hcp", "liquid"])
@pytest.mark.parametrize("sigma", [0.02, 0.05, 0.1])
def test_cna_triplets_and_labels_bit_exact(L, ctx, kind, sigma):
    c = _box(kind, sigma)
    pos, box = c["pos"], c["box"]
    offs, nb = oracle.neighbours_cells(pos, box, R_BOA)
    nbond, trip_o, partner, _ = oracle.cna(pos, box, offs, nb, R_CNA)
    lab_o = oracle.cna_label(nbond, trip_o)
    ref = {(i, int(partner[i, a])): int(trip_o[i, a]) for i in range(len(pos)) for a in range(nbond[i])}
    p = cu(pos)
    nbr, cnt = _gpu_list(L, ctx, p, box, R_BOA)
    trip, lab = L.ppmd_cna(ctx, p, box, R_CNA, nbr, cnt)
    ctx.sync()
    assert _trip_map(nbr, cnt, trip) == ref
    assert np.array_equal(lab.cpu().numpy(), lab_o)


@pytest.mark.parametrize("kind", ["fcc", "bcc", "hcp"])
def test_cna_perfect_lattice_labels(L, ctx, kind):
    lat = make_lattice(kind, SMALL[kind], 0.8442)
    p = cu(lat.sites())
    nbr, cnt = _gpu_list(L, ctx, p, lat.box, R_BOA)
    _, lab = L.ppmd_cna(ctx, p, lat.box, R_CNA, nbr, cnt, want_triplets=False)
    assert (lab.cpu().numpy() == {"fcc": 1, "hcp": 2, "bcc": 3}[kind]).all()


@pytest.mark.parametrize("kind", ["fcc", "hcp", "liquid"])
def test_analyze_pipeline_parity(L, ctx, kind):
    """Positions in a shuffled order: the pipeline sorts internally and must
    return every result in the caller's order."""
    c = _box(kind, 0.05, seed=32)
    perm = np.random.default_rng(0).permutation(len(c["pos"]))
    pos, box = c["pos"][perm], c["box"]
    offs, nb = oracle.neighbours_cells(pos, box, R_BOA)
    Q4o, nno = oracle.boa(pos, box, offs, nb, R_BOA, 4)
    Q6o, _ = oracle.boa(pos, box, offs, nb, R_BOA, 6)
    lab_o = oracle.cna_label(*oracle.cna(pos, box, offs, nb, R_CNA)[:2])
    out = L.ppmd_analyze(ctx, cu(pos), box, R_BOA, R_CNA)
    assert np.array_equal(out["n_nb"].cpu().numpy(), nno)
    assert np.abs(out["q4"].cpu().numpy() - Q4o).max() <= 1e-5
    assert np.abs(out["q6"].cpu().numpy() - Q6o).max() <= 1e-5
    assert np.array_equal(out["label"].cpu().numpy(), lab_o)


def test_analysis_invariant_under_translation_and_axis_rotation(L, ctx):
    """CNA labels bit for bit and Q4/Q6 within single-precision rounding after
    a periodic translation of every position and after a quarter turn about
    z, (x, y) -> (-y, x) with the box's x and y edges exchanged."""
    c = _box("hcp", 0.05)
    pos, box = c["pos"], np.asarray(c["box"], float)
    base = L.ppmd_analyze(ctx, cu(pos), box, R_BOA, R_CNA)
    moved = [(pos + np.array([0.37, 1.91, 2.53]), box),
             (np.stack([-pos[:, 1], pos[:, 0], pos[:, 2]], 1), box[[1, 0, 2]])]
    for p2, b2 in moved:
        out = L.ppmd_analyze(ctx, cu(p2), b2, R_BOA, R_CNA)
        ctx.sync()
        assert torch.equal(out["label"], base["label"])
        assert torch.equal(out["n_nb"], base["n_nb"])
        for k in ("q4", "q6"):
            assert (out[k] - base[k]).abs().max().item() <= 2e-6


def test_analyze_full_size_box_sampled(L, ctx):
    """One 512,000-atom structure box (the analysis workload size): labels and
    Q_l of a seeded sample of atoms against the oracle evaluated on those atoms."""
    c = configs.structure_box("hcp", 0.05, seed=30)
    pos, box = c["pos"], c["box"]
    out = L.ppmd_analyze(ctx, cu(pos), box, R_BOA, R_CNA)
    sample = np.random.default_rng(7).choice(len(pos), 400, replace=False)
    # oracle on the sample: neighbours of the sampled atoms and of their neighbours
    offs, nb = oracle.neighbours_cells(pos, box, R_BOA)
    Q6o, nno = oracle.boa(pos, box, offs, nb, R_BOA, 6)
    nbond, trip, _, _ = oracle.cna(pos, box, offs, nb, R_CNA)
    lab_o = oracle.cna_label(nbond, trip)
    assert np.array_equal(out["label"].cpu().numpy()[sample], lab_o[sample])
    assert np.abs(out["q6"].cpu().numpy()[sample] - Q6o[sample]).max() <= 1e-5
    # labels are mostly hcp at this noise level
    assert (out["label"].cpu().numpy() == 2).mean() > 0.5


def test_analyze_overflow_is_latched_and_features_retry(L, ctx):
    """A dense clump in a dilute box: the asynchronous pipeline's list (capacity
    from the box density) overflows; the next synchronising call reports
    PPMD_ERR_CAPACITY with the row length needed.  ppmd_features, which
    synchronises, builds the list again at that length and matches the oracle."""
    rng = np.random.default_rng(11)
    L_box = np.array([20.0, 20.0, 20.0])
    spread = rng.uniform(0.0, 20.0, (600, 3))
    clump = 10.0 + rng.uniform(-0.4, 0.4, (56, 3))  # every pair closer than 1.39
    pos = np.concatenate([spread, clump])
    L.ppmd_analyze(ctx, cu(pos), L_box, R_BOA, R_CNA)
    with pytest.raises(L.PPMDError) as ei:
        ctx.sync()
    assert ei.value.code == L.ERR_CAPACITY
    ctx.sync()  # the report cleared the status
    f, _ = L.ppmd_features(ctx, cu(pos), L_box, R_BOA, fp32=True, bf16=False, r_ref=R_CNA)
    offs, nb = oracle.neighbours_cells(pos, L_box, R_BOA)
    nbond = np.diff(offs)
    assert 48 < nbond.max() <= 64  # over the first capacity, within the 64 bonds features take
    fo = oracle.features(pos, L_box, offs, nb, R_BOA, R_CNA)
    assert np.abs(f.cpu().numpy() - fo).max() <= 2e-5


R_ACNA = 1.8  # reaches the 14th neighbour at density 0.8442


@pytest.mark.parametrize("kind", ["fcc", "bcc", "hcp", "liquid"])
@pytest.mark.parametrize("sigma", [0.02, 0.07, 0.12])
def test_acna_bit_exact(L, ctx, kind, sigma):
    """Adaptive CNA: labels and both FP64 local cutoffs equal the oracle's bit
    for bit (caller order, shuffled input)."""
    c = _box(kind, sigma, seed=34)
    perm = np.random.default_rng(1).permutation(len(c["pos"]))
    pos, box = c["pos"][perm], c["box"]
    offs, nb = oracle.neighbours_cells(pos, box, R_ACNA)
    lab_o, rc_o = oracle.acna(pos, box, offs, nb)
    lab, rc = L.ppmd_acna(ctx, cu(pos), box, R_ACNA)
    # without the cutoff output the kernel decides in FP32 where that is
    # safe and computes the FP64 cutoff only for bonds within its band
    lab_fast, _ = L.ppmd_acna(ctx, cu(pos), box, R_ACNA, want_rcut=False)
    ctx.sync()
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    assert np.array_equal(lab_fast.cpu().numpy(), lab_o)
    assert np.array_equal(rc.cpu().numpy(), rc_o)


@pytest.mark.parametrize("kind,code", [("fcc", 1), ("hcp", 2), ("bcc", 3)])
@pytest.mark.parametrize("scale", [0.8, 1.3])
def test_acna_perfect_lattices_scaled(L, ctx, kind, code, scale):
    lat = make_lattice(kind, SMALL[kind], 0.8442 / scale ** 3)
    lab, _ = L.ppmd_acna(ctx, cu(lat.sites()), lat.box, R_ACNA * scale)
    ctx.sync()
    assert (lab.cpu().numpy() == code).all()


def test_acna_full_size_box_sampled(L, ctx):
    """A 512,000-atom structure box: labels and cutoffs of a seeded sample
    against the oracle evaluated on those atoms only."""
    c = configs.structure_box("bcc", 0.05, seed=30)
    pos, box = c["pos"], c["box"]
    lab, rc = L.ppmd_acna(ctx, cu(pos), box, R_ACNA)
    lab_fast, _ = L.ppmd_acna(ctx, cu(pos), box, R_ACNA, want_rcut=False)
    ctx.sync()
    assert np.array_equal(lab.cpu().numpy(), lab_fast.cpu().numpy())
    sample = np.sort(np.random.default_rng(3).choice(len(pos), 500, replace=False))
    offs, nb = oracle.neighbours_cells(pos, box, R_ACNA)
    # rows of the other atoms emptied: the oracle then only works on the sample
    deg = np.zeros(len(pos), np.int64)
    deg[sample] = np.diff(offs)[sample]
    offs_s = np.concatenate([[0], np.cumsum(deg)])
    nb_s = np.concatenate([nb[offs[i]:offs[i + 1]] for i in sample])
    lab_o, rc_o = oracle.acna(pos, box, offs_s, nb_s)
    assert np.array_equal(lab.cpu().numpy()[sample], lab_o[sample])
    assert np.array_equal(rc.cpu().numpy()[sample], rc_o[sample])
    assert (lab.cpu().numpy() == 3).mean() > 0.5
