"""The Python binding checks every tensor it hands to the C library: the
element type, the shape the call reads or writes through the pointer,
contiguity, then CUDA memory as the pointers are taken.  A mismatch raises
ValueError before any pointer reaches the library (runs without a GPU: the
checks come before the context is used, and host tensors of the right type
and shape stop at the CUDA test)."""
from types import SimpleNamespace

import pytest
import torch


@pytest.fixture(scope="module")
def L():
    from paper_1704_03329_b300 import build
    build.build()
    from paper_1704_03329_b300 import lib
    return lib


BOX = [12.0, 12.0, 12.0]
# stands in for a Context: no call gets as far as using it
CTX = SimpleNamespace(h=None, check=lambda rc, allow_warn=True: rc)


def f64(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def i32(*shape):
    return torch.zeros(shape, dtype=torch.int32)


def _raises(fn, *words):
    with pytest.raises(ValueError) as ei:
        fn()
    msg = str(ei.value)
    for w in words:
        assert w in msg, msg


def test_positions_need_float64_rows_of_three(L):
    _raises(lambda: L.ppmd_build_cells(CTX, torch.zeros((5, 3), dtype=torch.float32), BOX, 2.8), "pos", "float64")
    _raises(lambda: L.ppmd_build_cells(CTX, f64(5, 4), BOX, 2.8), "pos", "shape")
    _raises(lambda: L.ppmd_build_cells(CTX, f64(15), BOX, 2.8), "pos", "shape")
    _raises(lambda: L.ppmd_lj_forces_cells(CTX, f64(5, 3).t().contiguous().t(), BOX), "pos", "contiguous")
    # right type and shape, host memory: refused as well
    _raises(lambda: L.ppmd_build_cells(CTX, f64(5, 3), BOX, 2.8), "CUDA")
    _raises(lambda: L.ppmd_acna(CTX, [[0.0, 0.0, 0.0]], BOX), "pos", "torch tensor")


def test_neighbour_tables_match_the_atoms(L):
    pos = f64(6, 3)
    _raises(lambda: L.ppmd_lj_forces(CTX, pos, BOX, i32(5, 8), i32(6)), "nbr", "[6, *]")
    _raises(lambda: L.ppmd_lj_forces(CTX, pos, BOX, i32(6, 8), i32(5)), "nbr_count", "[6]")
    _raises(lambda: L.ppmd_lj_forces(CTX, pos, BOX, i32(48), i32(6)), "nbr")
    _raises(lambda: L.ppmd_lj_forces(CTX, pos, BOX, torch.zeros((6, 8), dtype=torch.int64), i32(6)), "nbr", "int32")
    _raises(lambda: L.ppmd_boa_q46(CTX, pos, BOX, 1.5, i32(6, 8), torch.zeros(6, dtype=torch.int64)),
            "nbr_count", "int32")
    _raises(lambda: L.ppmd_cna(CTX, pos, BOX, 1.43, i32(7, 8), i32(6)), "nbr")
    _raises(lambda: L.ppmd_half_list(CTX, pos, BOX, i32(6, 8), i32(3)), "nbr_count")
    _raises(lambda: L.ppmd_lj_forces_newton3(CTX, pos, BOX, i32(6, 4), i32(2)), "half_count")
    # cell arrays of ppmd_build_cells: cell_start needs ncell + 1 entries
    _raises(lambda: L.ppmd_build_neighbours(CTX, pos, BOX, 2.8, i32(27), i32(6), [3, 3, 3], 8), "cell_start")
    _raises(lambda: L.ppmd_build_neighbours(CTX, pos, BOX, 2.8, i32(28), i32(5), [3, 3, 3], 8), "cell_atoms")


def test_particle_loops_check_every_array(L):
    _raises(lambda: L.ppmd_verlet_step(CTX, 1, f64(4, 3), f64(5, 3), f64(5, 3), BOX), "pos", "[5, 3]")
    _raises(lambda: L.ppmd_verlet_step(CTX, 1, f64(5, 3), f64(5, 3), f64(3, 5), BOX), "force")
    _raises(lambda: L.ppmd_kinetic_energy(CTX, torch.zeros((5, 3), dtype=torch.float32)), "vel", "float64")


def test_analysis_outputs_given_by_the_caller(L):
    pos = f64(6, 3)
    _raises(lambda: L.ppmd_analyze(CTX, pos, BOX, out={"q4": torch.zeros(5, dtype=torch.float32)}), "q4", "[6]")
    _raises(lambda: L.ppmd_analyze(CTX, pos, BOX, out={"label": i32(6)}), "label", "int8")
    _raises(lambda: L.ppmd_analyze(CTX, pos, BOX, out={"q8": torch.zeros(6, dtype=torch.float32)}), "q8")
    _raises(lambda: L.ppmd_analyze_boxes(CTX, pos, [0, 6], [BOX], out={"n_nb": f64(6)}), "n_nb", "int32")


def test_mlp_arrays(L):
    P = torch.zeros(L.MLP_NPARAM, dtype=torch.float32)
    x = torch.zeros((10, 32), dtype=torch.bfloat16)
    _raises(lambda: L.ppmd_mlp_forward(CTX, P[:-1], x), "params", f"[{L.MLP_NPARAM}]")
    _raises(lambda: L.ppmd_mlp_forward(CTX, P.double(), x), "params", "float32")
    _raises(lambda: L.ppmd_mlp_forward(CTX, P, x[:, :30].contiguous()), "x_bf16", "[*, 32]")
    _raises(lambda: L.ppmd_mlp_forward(CTX, P, x.float()), "x_bf16", "bfloat16")
    _raises(lambda: L.ppmd_mlp_grad(CTX, P, x, torch.zeros(9, dtype=torch.int8)), "y", "[10]")
    _raises(lambda: L.ppmd_mlp_grad(CTX, P, x, torch.zeros(10, dtype=torch.int64)), "y", "int8")
    _raises(lambda: L.ppmd_mlp_adamw(CTX, P, P, P[:100], P, 1), "v")
    _raises(lambda: L.ppmd_mlp_train_step(CTX, P, P, P, 1, x, torch.zeros(10, dtype=torch.int8),
                                          loss=torch.zeros(1, dtype=torch.float64)), "loss", "float32")
    _raises(lambda: L.ppmd_mlp_fit_input_norm(CTX, P, x.view(2, 5, 32)), "x_bf16")


def test_classifier_needs_parameters_in_mode_1(L):
    pos = f64(6, 3)
    _raises(lambda: L.ppmd_classify(CTX, pos, BOX, mode=1, params=None), "params", "required")
    _raises(lambda: L.ppmd_classify_boxes(CTX, pos, [0, 6], [BOX], mode=1,
                                          params=torch.zeros(L.MLP_NPARAM, dtype=torch.float64)), "params", "float32")
    # modes 0 and 2 take no parameters: the checks pass on to the CUDA test
    _raises(lambda: L.ppmd_classify(CTX, pos, BOX, mode=0), "CUDA")
    _raises(lambda: L.ppmd_classify(CTX, pos, BOX, mode=2), "CUDA")


def test_integrator_state_and_energy_rows(L):
    md = object.__new__(L.MD)  # the checks need only the atom count
    md.n, md.h, md.ctx = 8, None, CTX
    _raises(lambda: md.set_state(f64(7, 3), f64(8, 3)), "pos", "[8, 3]")
    _raises(lambda: md.set_state(f64(8, 3), torch.zeros((8, 3), dtype=torch.float32)), "vel", "float64")
    _raises(lambda: md.set_state(f64(8, 3), None), "vel", "required")
    _raises(lambda: md.get_state(None, f64(8, 2)), "vel")
    _raises(lambda: md.get_state(None, None, f64(8, 3)), "CUDA")
    # a row per step: energies [nsteps][2], qrows [nsteps][3]
    _raises(lambda: md.run(10, f64(9, 2)), "energies", "20")
    _raises(lambda: md.run_analysed(10, None, f64(10, 2)), "qrows", "30")
    _raises(lambda: md.run(10, f64(10, 2)), "CUDA")


def test_allocation_free_forces_check_their_arrays(L):
    """ppmd_lj_forces_noalloc takes every array from the caller: positions
    float64 [n][3], forces of the same shape, an int32 list of n rows and
    counts; an n above the static limit is the one override it accepts
    (refused by the library before anything runs)."""
    pos, F = f64(6, 3), f64(6, 3)
    nbr, cnt = i32(6, 8), i32(6)
    st = SimpleNamespace(cuda_stream=0)  # no call gets as far as the stream

    def call(*a, **kw):
        return lambda: L.ppmd_lj_forces_noalloc(*a, stream=st, **kw)
    _raises(call(pos.float(), BOX, nbr, cnt, F, None, None), "pos")
    _raises(call(pos, BOX, nbr, cnt, f64(5, 3), None, None), "force")
    _raises(call(pos, BOX, i32(5, 8), cnt, F, None, None), "nbr")
    _raises(call(pos, BOX, nbr, i32(5), F, None, None), "nbr_count")
    _raises(call(pos, BOX, nbr, cnt, F, f64(5), None), "e_atom")
    _raises(call(pos, BOX, nbr, cnt, F, None, f64(1)), "totals")
    # an n at or below the limit is taken from the arrays, never from the caller
    _raises(call(pos, BOX, nbr, cnt, F.float(), None, None, n=3), "force")
