"""The seeded synthetic workloads keep the sizes and shapes the benchmark and
the full-size parity tests are stated for (a change to a generator would
otherwise change what is measured without notice), and generation is
deterministic."""
import numpy as np

from synth import configs


def test_lj_solid_is_the_million_atom_fcc_box():
    c = configs.lj_solid()
    assert len(c["pos"]) == 4 * 63 ** 3 == 1000188
    assert np.allclose(c["box"], 105.8146, atol=5e-5)
    assert (c["rc"], c["r_list"], c["rebuild_every"]) == (2.5, 2.8, 10)
    assert np.abs(c["vel"].sum(0)).max() < 1e-9  # no centre-of-mass drift
    assert ((c["pos"] >= 0) & (c["pos"] < c["box"])).all()


def test_replicas_total_and_ranges():
    reps = configs.replicas()
    n = np.array([len(r["pos"]) for r in reps])
    assert len(reps) == 256 and n.sum() == 2034923
    assert n.min() >= 500 and n.max() <= 32000
    for r in reps:
        rho = len(r["pos"]) / np.prod(r["box"])
        assert 0.7 - 1e-9 <= rho <= 1.0 + 1e-9
        assert 2.5 <= r["r_list"] <= 2.8 and (r["box"] / r["r_list"] >= 3.0 - 1e-12).all()


def test_otf_box_is_the_papers_weak_scaling_size():
    c = configs.otf_box()
    assert len(c["pos"]) == 524288
    assert np.isclose(len(c["pos"]) / np.prod(c["box"]), 0.8442)
    assert (c["rc"], c["r_list"], c["rebuild_every"]) == (3.0, 3.3, 18)


def test_structure_box_size_and_determinism():
    a = configs.structure_box("fcc", 0.05, seed=30)
    assert len(a["pos"]) == 512000
    b = configs.lj_solid(n_cells=6)
    c = configs.lj_solid(n_cells=6)
    assert np.array_equal(b["pos"], c["pos"]) and np.array_equal(b["vel"], c["vel"])


def test_liquid_boxes_are_tiled_equilibrated_snapshots():
    """The liquid boxes: copies of an LJ liquid snapshot (the oracle's run at
    density 0.8442, T 1.5; oracle/make_liquid.py) at the boxes' sizes, at the
    workload density, with no pair within 1e-6 of the analysis cutoffs; the
    classifier's training and inference sets see different snapshots."""
    from synth.configs import R_BOA, R_CNA
    a = configs.structure_box("liquid", 0.05, seed=30)
    assert len(a["pos"]) == 512000
    assert np.isclose(len(a["pos"]) / np.prod(a["box"]), 0.8442, rtol=1e-12)
    tr = configs.structure_box("liquid", 0.05, seed=50003, cells=configs.CLASSIFIER_CELLS["liquid"])
    te = configs.structure_box("liquid", 0.05, seed=51003, cells=configs.CLASSIFIER_CELLS["liquid"])
    assert len(tr["pos"]) == len(te["pos"]) == 128000
    assert not np.array_equal(tr["pos"], te["pos"])
    s = configs.structure_box("liquid", 0.0, seed=41, cells=(12, 12, 12))
    assert len(s["pos"]) == 1728
    from synth.lattices import min_pair_margin
    assert min_pair_margin(s["pos"], s["box"], (R_BOA, R_CNA)) >= 1e-6
    # a liquid: no long-range order, so no lattice site holds an atom for
    # long; the nearest-neighbour distances spread well beyond a crystal's
    d = s["pos"][:, None, :] - s["pos"][None, :, :]
    d -= s["box"] * np.rint(d / s["box"])
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    nn = r.min(1)
    assert nn.std() > 0.03 and 0.85 < nn.mean() < 1.15
