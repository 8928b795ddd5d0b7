"""Thin ctypes binding of libppmd.so (include/ppmd.h).

Only argument marshalling lives here: every step of the computation runs in
the library's CUDA kernels.  Tensors are PyTorch CUDA tensors (device memory
and streams); there is no CPU fallback -- importing this module fails if the
compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libppmd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1704_03329_b300.build` "
                      "(there is no CPU fallback)")

_lib = C.CDLL(LIB_PATH)

OK, ERR_INVALID, ERR_BOX, ERR_CAPACITY, ERR_NONFINITE, ERR_CUDA, ERR_TIMEOUT, ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6, -7
WARN_SKIN = 1
FP64, FP32 = 0, 1
PAIR_COLUMNS, PAIR_BRICKS = 0, 1
MD_SHAPES = 8  # launch shapes of ppmd_md_set_shape / ppmd_md_tune
OTHER, FCC, HCP, BCC = 0, 1, 2, 3
_NAMES = {0: "PPMD_OK", -1: "PPMD_ERR_INVALID", -2: "PPMD_ERR_BOX", -3: "PPMD_ERR_CAPACITY",
          -4: "PPMD_ERR_NONFINITE", -5: "PPMD_ERR_CUDA", -6: "PPMD_ERR_TIMEOUT", -7: "PPMD_ERR_NOMEM",
          1: "PPMD_WARN_SKIN"}


class Box(C.Structure):
    _fields_ = [("L", C.c_double * 3)]


class LJParams(C.Structure):
    _fields_ = [("eps", C.c_double), ("sigma", C.c_double), ("rc", C.c_double), ("shift", C.c_double)]


class MDParams(C.Structure):
    _fields_ = [("lj", LJParams), ("r_list", C.c_double), ("mass", C.c_double), ("dt", C.c_double),
                ("rebuild_every", C.c_int32), ("max_nbr", C.c_int32), ("prec", C.c_int32),
                ("energy_every", C.c_int32)]


class PPMDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_P, _I64, _I32, _D, _I = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_int
_SIGS = {
    "ppmd_create": (_I, [C.POINTER(_P), _I, _P]),
    "ppmd_destroy": (_I, [_P]),
    "ppmd_set_stream": (_I, [_P, _P]),
    "ppmd_sync": (_I, [_P]),
    "ppmd_status": (_I, [_P, C.POINTER(_I64)]),
    "ppmd_last_error": (C.c_char_p, [_P]),
    "ppmd_kernel_count": (_I64, [_P]),
    "ppmd_build_cells": (_I, [_P, _P, _I64, C.POINTER(Box), _D, _P, _P, _P, C.POINTER(_I32), _I64]),
    "ppmd_build_neighbours": (_I, [_P, _P, _I64, C.POINTER(Box), _D, _P, _P, C.POINTER(_I32), _P, _P, _I32,
                                   C.POINTER(_I32)]),
    "ppmd_lj_forces": (_I, [_P, _P, _I64, C.POINTER(Box), C.POINTER(LJParams), _P, _P, _I32, _I, _P, _P, _P, _P]),
    "ppmd_lj_forces_cells": (_I, [_P, _P, _I64, C.POINTER(Box), C.POINTER(LJParams), _I, _P, _P, _P, _P]),
    "ppmd_half_list": (_I, [_P, _P, _I64, C.POINTER(Box), _P, _P, _I32, _P, _P, _I32]),
    "ppmd_lj_forces_newton3": (_I, [_P, _P, _I64, C.POINTER(Box), C.POINTER(LJParams), _P, _P, _I32, _I, _P, _P, _P,
                                    _P]),
    "ppmd_verlet_step": (_I, [_P, _I, _P, _P, _P, _I64, C.POINTER(Box), _D, _D]),
    "ppmd_kinetic_energy": (_I, [_P, _P, _I64, _D, _P]),
    "ppmd_boa_q46": (_I, [_P, _P, _I64, C.POINTER(Box), _D, _P, _P, _I32, _P, _P, _P]),
    "ppmd_cna": (_I, [_P, _P, _I64, C.POINTER(Box), _D, _P, _P, _I32, _P, _P]),
    "ppmd_analyze": (_I, [_P, _P, _I64, C.POINTER(Box), _D, _D, _P, _P, _P, _P]),
    "ppmd_features": (_I, [_P, _P, _I64, C.POINTER(Box), _D, _D, _P, _P]),
    "ppmd_mlp_forward": (_I, [_P, _P, _P, _I64, _P]),
    "ppmd_acna": (_I, [_P, _P, _I64, C.POINTER(Box), _D, _P, _P]),
    "ppmd_md_set_thermostat": (_I, [_P, _D, _D, C.c_uint64]),
    "ppmd_md_set_boa": (_I, [_P, C.c_int32, _D]),
    "ppmd_md_run_analysed": (_I, [_P, C.c_int32, _P, _P, C.c_int]),
    "ppmd_md_get_q": (_I, [_P, _P, _P, _P]),
    "ppmd_mlp_fit_input_norm": (_I, [_P, _P, _P, _I64]),
    "ppmd_mlp_grad": (_I, [_P, _P, _P, _P, _I64, _P, _P]),
    "ppmd_mlp_adamw": (_I, [_P, _P, _P, _P, _P, _I64, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float]),
    "ppmd_mlp_train_step": (_I, [_P, _P, _P, _P, _I64, _P, _P, _I64, C.c_float, C.c_float, _P]),
    "ppmd_classify": (_I, [_P, _I, _P, _I64, C.POINTER(Box), _D, _D, _P, C.c_float, _P, _P, C.POINTER(_I64)]),
    "ppmd_analyze_boxes": (_I, [_P, _P, _I64, _P, _P, _D, _D, _P, _P, _P, _P]),
    "ppmd_classify_boxes": (_I, [_P, _I, _P, _I64, _P, _P, _D, _D, _P, C.c_float, _P, _P, C.POINTER(_I64)]),
    "ppmd_md_create": (_I, [_P, C.POINTER(_P), _I64, _P, _P, _P, C.POINTER(MDParams)]),
    "ppmd_md_destroy": (_I, [_P]),
    "ppmd_md_set_state": (_I, [_P, _P, _P]),
    "ppmd_md_run": (_I, [_P, _I32, _P, _I]),
    "ppmd_md_get_state": (_I, [_P, _P, _P, _P]),
    "ppmd_md_info": (_I, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_D)]),
    "ppmd_md_forces": (_I, [_P]),
    "ppmd_md_list_stats": (_I, [_P, C.POINTER(_I64), C.POINTER(_I32)]),
    "ppmd_md_get_list": (_I, [_P, _P, _P, _I32]),
    "ppmd_md_set_pair_loop": (_I, [_P, _I]),
    "ppmd_md_set_check": (_I, [_P, _I]),
    "ppmd_md_missed_pairs": (_I, [_P, C.POINTER(_I64)]),
    "ppmd_md_time_pair_loops": (_I, [_P, _I]),
    "ppmd_md_pair_loop_times": (_I, [_P, C.POINTER(_D), C.POINTER(_I32), C.POINTER(_D), C.POINTER(_I32)]),
    "ppmd_md_set_shape": (_I, [_P, _I32]),
    "ppmd_md_get_shape": (_I, [_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)]),
    "ppmd_md_tune": (_I, [_P, _I32, C.c_char_p, C.POINTER(_I32), C.POINTER(_D), C.POINTER(_I)]),
    "ppmd_lj_forces_noalloc": (_I, [_P, _P, _I64, C.POINTER(Box), C.POINTER(LJParams), _P, _P, _I32, _I, _P, _P, _P,
                                    _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_symbols():
    return list(_SIGS)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _need(t, name, dtype, shape=None, numel=None, optional=False):
    """Check a tensor argument against what the C call reads or writes
    through its pointer, before any pointer is taken: the element type, the
    shape (None entries: any extent) or at least `numel` elements, and a
    contiguous layout (_ptr then requires CUDA memory).  A mismatch raises
    ValueError rather than letting a kernel run past the end of the buffer."""
    if t is None:
        if optional:
            return
        raise ValueError(f"{name}: a tensor is required")
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if shape is not None:
        if t.dim() != len(shape) or any(s is not None and t.shape[k] != s for k, s in enumerate(shape)):
            want = "[" + ", ".join("*" if s is None else str(s) for s in shape) + "]"
            raise ValueError(f"{name}: expected shape {want}, got {list(t.shape)}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name}: expected at least {numel} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")


def _positions(t, name="pos"):
    """A float64 [n][3] position or velocity array; returns n."""
    _need(t, name, torch.float64, (None, 3))
    return t.shape[0]


def _rows(nbr, name, n):
    """An int32 neighbour table [n][max_nbr]; returns max_nbr."""
    _need(nbr, name, torch.int32, (n, None))
    return nbr.shape[1]


def _box(L):
    b = Box()
    for d in range(3):
        b.L[d] = float(L[d])
    return b


class Context:
    """A library context bound to a CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        torch.cuda.init()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self.device = device
        h = _P()
        rc = _lib.ppmd_create(C.byref(h), int(device), C.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PPMDError(rc, "ppmd_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib.ppmd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc, allow_warn=True):
        if rc < 0 or (rc > 0 and not allow_warn):
            raise PPMDError(rc, _lib.ppmd_last_error(self.h).decode(errors="replace"))
        return rc

    def sync(self):
        return self.check(_lib.ppmd_sync(self.h))

    def status(self):
        nd = _I64()
        rc = _lib.ppmd_status(self.h, C.byref(nd))
        return rc, nd.value

    def kernel_count(self) -> int:
        return int(_lib.ppmd_kernel_count(self.h))

    def last_error(self) -> str:
        return _lib.ppmd_last_error(self.h).decode(errors="replace")


def ppmd_build_cells(ctx: Context, pos, box, min_cell_width, cell_capacity=None):
    """Cell list; returns (ncell[3] list, cell_of, cell_start, cell_atoms) as int32 CUDA tensors."""
    n = _positions(pos)
    dev = pos.device
    ncell = [max(1, int(float(box[d]) // float(min_cell_width))) for d in range(3)]
    cap = cell_capacity if cell_capacity is not None else ncell[0] * ncell[1] * ncell[2] + 1
    cell_of = torch.empty(n, dtype=torch.int32, device=dev)
    cell_start = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    cell_atoms = torch.empty(n, dtype=torch.int32, device=dev)
    nc = (_I32 * 3)()
    b = _box(box)
    rc = _lib.ppmd_build_cells(ctx.h, _ptr(pos), n, C.byref(b), float(min_cell_width), _ptr(cell_of), _ptr(cell_start),
                               _ptr(cell_atoms), nc, int(cap))
    ctx.check(rc)
    nc = [nc[0], nc[1], nc[2]]
    return nc, cell_of, cell_start[: nc[0] * nc[1] * nc[2] + 1], cell_atoms


def ppmd_build_neighbours(ctx: Context, pos, box, r_list, cell_start, cell_atoms, ncell, max_nbr, want_needed=False):
    """Neighbour list rows nbr[n, max_nbr] (int32) and counts nbr_count[n]."""
    n = _positions(pos)
    ncell = [int(x) for x in ncell]
    _need(cell_start, "cell_start", torch.int32, numel=ncell[0] * ncell[1] * ncell[2] + 1)
    _need(cell_atoms, "cell_atoms", torch.int32, (n,))
    nbr = torch.empty((n, max_nbr), dtype=torch.int32, device=pos.device)
    cnt = torch.empty(n, dtype=torch.int32, device=pos.device)
    nc = (_I32 * 3)(*[int(x) for x in ncell])
    needed = _I32(0)
    b = _box(box)
    rc = _lib.ppmd_build_neighbours(ctx.h, _ptr(pos), n, C.byref(b), float(r_list), _ptr(cell_start), _ptr(cell_atoms),
                                    nc, _ptr(nbr), _ptr(cnt), int(max_nbr),
                                    C.byref(needed) if want_needed else None)
    ctx.check(rc)
    if want_needed:
        return nbr, cnt, needed.value
    return nbr, cnt


def ppmd_lj_forces(ctx: Context, pos, box, nbr, nbr_count, rc=2.5, eps=1.0, sigma=1.0, shift=0.0, prec=FP32,
                   want_energy=True):
    """Forces [n,3] f64, per-atom energies [n] f64, and device scalars (U, W)."""
    n = _positions(pos)
    max_nbr = _rows(nbr, "nbr", n)
    _need(nbr_count, "nbr_count", torch.int32, (n,))
    dev = pos.device
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev) if want_energy else None
    tot = torch.zeros(2, dtype=torch.float64, device=dev)
    p = LJParams(eps, sigma, rc, shift)
    b = _box(box)
    code = _lib.ppmd_lj_forces(ctx.h, _ptr(pos), n, C.byref(b), C.byref(p), _ptr(nbr), _ptr(nbr_count), int(max_nbr),
                               int(prec), _ptr(F), _ptr(e) if e is not None else None, _ptr(tot[0:1]),
                               C.c_void_p(tot.data_ptr() + 8))
    ctx.check(code)
    return F, e, tot


def ppmd_lj_forces_cells(ctx: Context, pos, box, rc=2.5, eps=1.0, sigma=1.0, shift=0.0, prec=FP32, want_energy=True):
    """List-free pair loop (cells of edge >= rc swept directly, no neighbour
    list): forces [n,3] f64, per-atom energies [n] f64, device scalars (U, W)."""
    n = _positions(pos)
    dev = pos.device
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev) if want_energy else None
    tot = torch.zeros(2, dtype=torch.float64, device=dev)
    p = LJParams(eps, sigma, rc, shift)
    b = _box(box)
    code = _lib.ppmd_lj_forces_cells(ctx.h, _ptr(pos), n, C.byref(b), C.byref(p), int(prec), _ptr(F),
                                     _ptr(e) if e is not None else None, _ptr(tot[0:1]), C.c_void_p(tot.data_ptr() + 8))
    ctx.check(code)
    return F, e, tot


def ppmd_half_list(ctx: Context, pos, box, nbr, nbr_count, max_half=None):
    """Half list of a full row-major list [n, max_nbr]: each pair kept by the
    atom from which the other lies in the upper half space (z, y, x order)."""
    n = _positions(pos)
    max_nbr = _rows(nbr, "nbr", n)
    _need(nbr_count, "nbr_count", torch.int32, (n,))
    max_half = (max_nbr + 1) // 2 + 8 if max_half is None else max_half
    half = torch.empty((n, max_half), dtype=torch.int32, device=nbr.device)
    hcnt = torch.empty(n, dtype=torch.int32, device=nbr.device)
    b = _box(box)
    ctx.check(_lib.ppmd_half_list(ctx.h, _ptr(pos), n, C.byref(b), _ptr(nbr), _ptr(nbr_count), int(max_nbr), _ptr(half),
                                  _ptr(hcnt), int(max_half)))
    return half, hcnt


def ppmd_lj_forces_newton3(ctx: Context, pos, box, half, half_count, rc=2.5, eps=1.0, sigma=1.0, shift=0.0, prec=FP32,
                           want_energy=True):
    """Forces [n,3] f64, per-atom energies [n] f64 and device scalars (U, W)
    from a half list (each pair once, Newton's third law)."""
    n = _positions(pos)
    _rows(half, "half", n)
    _need(half_count, "half_count", torch.int32, (n,))
    dev = pos.device
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev) if want_energy else None
    tot = torch.zeros(2, dtype=torch.float64, device=dev)
    p = LJParams(eps, sigma, rc, shift)
    b = _box(box)
    max_half = half.shape[1] if half.dim() == 2 else 0
    ctx.check(_lib.ppmd_lj_forces_newton3(ctx.h, _ptr(pos), n, C.byref(b), C.byref(p), _ptr(half), _ptr(half_count),
                                          int(max_half), int(prec), _ptr(F), _ptr(e) if e is not None else None,
                                          _ptr(tot[0:1]), C.c_void_p(tot.data_ptr() + 8)))
    return F, e, tot


def ppmd_verlet_step(ctx: Context, phase, pos, vel, force, box, mass=1.0, dt=0.005):
    n = _positions(vel, "vel")
    _need(pos, "pos", torch.float64, (n, 3))
    _need(force, "force", torch.float64, (n, 3))
    b = _box(box)
    ctx.check(_lib.ppmd_verlet_step(ctx.h, int(phase), _ptr(pos), _ptr(vel), _ptr(force), vel.shape[0], C.byref(b),
                                    float(mass), float(dt)))


def ppmd_kinetic_energy(ctx: Context, vel, mass=1.0):
    _positions(vel, "vel")
    ke = torch.zeros(1, dtype=torch.float64, device=vel.device)
    ctx.check(_lib.ppmd_kinetic_energy(ctx.h, _ptr(vel), vel.shape[0], float(mass), _ptr(ke)))
    return ke


def _opt(t):
    return _ptr(t) if t is not None else None


def ppmd_boa_q46(ctx: Context, pos, box, r_cut, nbr, nbr_count):
    """Q4, Q6 (float32 [n]) and bonded-neighbour counts (int32 [n])."""
    n = _positions(pos)
    _rows(nbr, "nbr", n)
    _need(nbr_count, "nbr_count", torch.int32, (n,))
    q4 = torch.empty(n, dtype=torch.float32, device=pos.device)
    q6 = torch.empty(n, dtype=torch.float32, device=pos.device)
    nnb = torch.empty(n, dtype=torch.int32, device=pos.device)
    b = _box(box)
    ctx.check(_lib.ppmd_boa_q46(ctx.h, _ptr(pos), n, C.byref(b), float(r_cut), _ptr(nbr), _ptr(nbr_count),
                                int(nbr.shape[1]), _ptr(q4), _ptr(q6), _ptr(nnb)))
    return q4, q6, nnb


def ppmd_cna(ctx: Context, pos, box, r_cut, nbr, nbr_count, want_triplets=True):
    """CNA triplets (uint32 as int32 [n, max_nbr]) and labels (int8 [n])."""
    n = _positions(pos)
    _rows(nbr, "nbr", n)
    _need(nbr_count, "nbr_count", torch.int32, (n,))
    trip = torch.empty(nbr.shape, dtype=torch.int32, device=pos.device) if want_triplets else None
    lab = torch.empty(n, dtype=torch.int8, device=pos.device)
    b = _box(box)
    ctx.check(_lib.ppmd_cna(ctx.h, _ptr(pos), n, C.byref(b), float(r_cut), _ptr(nbr), _ptr(nbr_count),
                            int(nbr.shape[1]), _opt(trip), _ptr(lab)))
    return trip, lab


def ppmd_analyze(ctx: Context, pos, box, r_boa=1.5, r_cna=None, boa=True, cna=True, out=None):
    """Pipeline from positions; returns dict with q4, q6, n_nb and/or label."""
    n = _positions(pos)
    out = _analysis_outputs(out, n, pos.device, boa, cna)
    b = _box(box)
    ctx.check(_lib.ppmd_analyze(ctx.h, _ptr(pos), n, C.byref(b), float(r_boa or 0.0), float(r_cna or 0.0),
                                _opt(out.get("q4")), _opt(out.get("q6")), _opt(out.get("n_nb")),
                                _opt(out.get("label"))))
    return out


_OUT_TYPES = {"q4": torch.float32, "q6": torch.float32, "n_nb": torch.int32, "label": torch.int8}


def _analysis_outputs(out, n, dev, boa, cna):
    """The output dict of ppmd_analyze(_boxes): the caller's tensors (checked:
    one element per atom of the right type) and new ones for the rest."""
    out = out or {}
    for k, t in out.items():
        if k not in _OUT_TYPES:
            raise ValueError(f"out: unknown key {k!r} (expected q4, q6, n_nb, label)")
        _need(t, f"out[{k!r}]", _OUT_TYPES[k], (n,))
    for k in (("q4", "q6", "n_nb") if boa else ()) + (("label",) if cna else ()):
        out.setdefault(k, torch.empty(n, dtype=_OUT_TYPES[k], device=dev))
    return out


def _box_set(atom_off, boxes):
    """Host tables of a box set: int64 offsets [nbox + 1] and the boxes."""
    nbox = len(atom_off) - 1
    off = (C.c_int64 * (nbox + 1))(*[int(x) for x in atom_off])
    bx = (Box * max(nbox, 1))()
    for b in range(nbox):
        for d in range(3):
            bx[b].L[d] = float(boxes[b][d])
    return nbox, off, bx


def ppmd_analyze_boxes(ctx: Context, pos, atom_off, boxes, r_boa=1.5, r_cna=None, boa=True, cna=True, out=None):
    """ppmd_analyze over several independent boxes (box b: atoms atom_off[b] ..
    atom_off[b + 1] - 1 of pos) in one pipeline; same outputs over all atoms."""
    n = _positions(pos)
    out = _analysis_outputs(out, n, pos.device, boa, cna)
    nbox, off, bx = _box_set(atom_off, boxes)
    if off[nbox] != n:
        raise ValueError("atom_off[-1] must equal the number of atoms")
    ctx.check(_lib.ppmd_analyze_boxes(ctx.h, _ptr(pos), nbox, C.cast(off, _P), C.cast(bx, _P), float(r_boa or 0.0),
                                      float(r_cna or 0.0), _opt(out.get("q4")), _opt(out.get("q6")),
                                      _opt(out.get("n_nb")), _opt(out.get("label"))))
    return out


def ppmd_acna(ctx: Context, pos, box, r_list=1.8, want_rcut=True):
    """Adaptive CNA labels int8 [n] and the local cutoffs float64 [n, 2] (caller order)."""
    n = _positions(pos)
    lab = torch.empty(n, dtype=torch.int8, device=pos.device)
    rc = torch.empty((n, 2), dtype=torch.float64, device=pos.device) if want_rcut else None
    b = _box(box)
    ctx.check(_lib.ppmd_acna(ctx.h, _ptr(pos), n, C.byref(b), float(r_list), _ptr(lab), _opt(rc)))
    return lab, rc


MLP_NPARAM = 6464


def ppmd_features(ctx: Context, pos, box, r_feat=1.5, fp32=True, bf16=False, r_ref=1.433625):
    """Classifier features: float32 [n, 30] and/or bfloat16 [n, 32] (caller order)."""
    n = _positions(pos)
    f = torch.empty((n, 30), dtype=torch.float32, device=pos.device) if fp32 else None
    fb = torch.empty((n, 32), dtype=torch.bfloat16, device=pos.device) if bf16 else None
    b = _box(box)
    ctx.check(_lib.ppmd_features(ctx.h, _ptr(pos), n, C.byref(b), float(r_feat), float(r_ref), _opt(f), _opt(fb)))
    return f, fb


def _mlp_params(t, name="params"):
    _need(t, name, torch.float32, (MLP_NPARAM,))


def _mlp_rows(x):
    """BF16 feature rows [n][32] (30 used); returns n."""
    _need(x, "x_bf16", torch.bfloat16, (None, 32))
    return x.shape[0]


def ppmd_mlp_fit_input_norm(ctx: Context, params, x_bf16):
    _mlp_params(params)
    _mlp_rows(x_bf16)
    ctx.check(_lib.ppmd_mlp_fit_input_norm(ctx.h, _ptr(params), _ptr(x_bf16), x_bf16.shape[0]))


def ppmd_mlp_forward(ctx: Context, params, x_bf16):
    _mlp_params(params)
    n = _mlp_rows(x_bf16)
    logits = torch.empty((n, 4), dtype=torch.float32, device=x_bf16.device)
    ctx.check(_lib.ppmd_mlp_forward(ctx.h, _ptr(params), _ptr(x_bf16), n, _ptr(logits)))
    return logits


def ppmd_mlp_grad(ctx: Context, params, x_bf16, y):
    _mlp_params(params)
    _need(y, "y", torch.int8, (_mlp_rows(x_bf16),))
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    ctx.check(_lib.ppmd_mlp_grad(ctx.h, _ptr(params), _ptr(x_bf16), _ptr(y), x_bf16.shape[0], _ptr(grad), _ptr(loss)))
    return grad, loss


def ppmd_mlp_adamw(ctx: Context, params, m, v, grad, step, lr=1e-3, wd=0.01, beta1=0.9, beta2=0.999, eps=1e-8):
    for t, name in ((params, "params"), (m, "m"), (v, "v"), (grad, "grad")):
        _mlp_params(t, name)
    ctx.check(_lib.ppmd_mlp_adamw(ctx.h, _ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step), lr, wd, beta1, beta2,
                                  eps))


def ppmd_mlp_train_step(ctx: Context, params, m, v, step, x_bf16, y, lr=1e-3, wd=0.01, loss=None):
    for t, name in ((params, "params"), (m, "m"), (v, "v")):
        _mlp_params(t, name)
    _need(y, "y", torch.int8, (_mlp_rows(x_bf16),))
    _need(loss, "loss", torch.float32, numel=1, optional=True)
    ctx.check(_lib.ppmd_mlp_train_step(ctx.h, _ptr(params), _ptr(m), _ptr(v), int(step), _ptr(x_bf16), _ptr(y),
                                       x_bf16.shape[0], lr, wd, _opt(loss)))


def ppmd_classify(ctx: Context, pos, box, mode=1, params=None, threshold=0.9, r_feat=1.5, r_cna=1.433625,
                  want_confidence=True, count=True):
    """Labels int8 [n], confidence float32 [n] (mode 1; mode 2: the distance to
    the nearest table (Q4, Q6), with threshold the tolerance), number of CNA
    fallbacks (None with count=False: the call is then asynchronous)."""
    n = _positions(pos)
    _need(params, "params", torch.float32, (MLP_NPARAM,), optional=mode != 1)
    lab = torch.empty(n, dtype=torch.int8, device=pos.device)
    conf = torch.empty(n, dtype=torch.float32, device=pos.device) if (want_confidence and mode in (1, 2)) else None
    nfb = _I64(0)
    b = _box(box)
    ctx.check(_lib.ppmd_classify(ctx.h, int(mode), _ptr(pos), n, C.byref(b), float(r_feat), float(r_cna), _opt(params),
                                 float(threshold), _ptr(lab), _opt(conf), C.byref(nfb) if count else None))
    return lab, conf, (nfb.value if count else None)


def ppmd_classify_boxes(ctx: Context, pos, atom_off, boxes, mode=1, params=None, threshold=0.9, r_feat=1.5,
                        r_cna=1.433625, want_confidence=True, count=True):
    """ppmd_classify over several independent boxes in one pipeline (box set as
    ppmd_analyze_boxes); labels, confidences and the total fallback count."""
    n = _positions(pos)
    _need(params, "params", torch.float32, (MLP_NPARAM,), optional=mode != 1)
    lab = torch.empty(n, dtype=torch.int8, device=pos.device)
    conf = torch.empty(n, dtype=torch.float32, device=pos.device) if (want_confidence and mode in (1, 2)) else None
    nfb = _I64(0)
    nbox, off, bx = _box_set(atom_off, boxes)
    if off[nbox] != n:
        raise ValueError("atom_off[-1] must equal the number of atoms")
    ctx.check(_lib.ppmd_classify_boxes(ctx.h, int(mode), _ptr(pos), nbox, C.cast(off, _P), C.cast(bx, _P), float(r_feat),
                                       float(r_cna), _opt(params), float(threshold), _ptr(lab), _opt(conf),
                                       C.byref(nfb) if count else None))
    return lab, conf, (nfb.value if count else None)


class MD:
    """Time stepping of one box or a batch of boxes (ppmd_md_*)."""

    def __init__(self, ctx: Context, atom_off, boxes, r_list=2.8, rc=2.5, eps=1.0, sigma=1.0, shift=0.0, mass=1.0,
                 dt=0.005, rebuild_every=10, max_nbr=128, prec=FP32, energy_every=0, box_r_list=None):
        self.ctx = ctx
        off = (C.c_int64 * len(atom_off))(*[int(x) for x in atom_off])
        nbox = len(atom_off) - 1
        bx = (Box * nbox)()
        for b in range(nbox):
            for d in range(3):
                bx[b].L[d] = float(boxes[b][d])
        brl = None
        if box_r_list is not None:
            brl = (C.c_double * nbox)(*[float(x) for x in box_r_list])
        p = MDParams(LJParams(eps, sigma, rc, shift), r_list, mass, dt, rebuild_every, max_nbr, prec, energy_every)
        h = _P()
        code = _lib.ppmd_md_create(ctx.h, C.byref(h), nbox, C.cast(off, _P), C.cast(bx, _P),
                                   C.cast(brl, _P) if brl is not None else None, C.byref(p))
        ctx.check(code)
        self.h = h
        self.n = int(atom_off[-1])
        self.params = p

    def close(self):
        if getattr(self, "h", None):
            # a context destroyed first (objects collected together at exit)
            # has taken the device state with it: nothing left to release
            if getattr(self.ctx, "h", None):
                _lib.ppmd_md_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, pos, vel):
        _need(pos, "pos", torch.float64, (self.n, 3))
        _need(vel, "vel", torch.float64, (self.n, 3))
        self.ctx.check(_lib.ppmd_md_set_state(self.h, _ptr(pos), _ptr(vel)))

    def run(self, nsteps, energies=None, use_graph=True):
        _need(energies, "energies", torch.float64, numel=2 * int(nsteps), optional=True)
        self.ctx.check(_lib.ppmd_md_run(self.h, int(nsteps), _ptr(energies) if energies is not None else None,
                                        1 if use_graph else 0))

    def set_thermostat(self, T, nu, seed):
        self.ctx.check(_lib.ppmd_md_set_thermostat(self.h, float(T), float(nu), int(seed)))

    def set_boa(self, every, r_boa=1.5):
        self.ctx.check(_lib.ppmd_md_set_boa(self.h, int(every), float(r_boa)))

    def run_analysed(self, nsteps, energies=None, qrows=None, use_graph=True):
        _need(energies, "energies", torch.float64, numel=2 * int(nsteps), optional=True)
        _need(qrows, "qrows", torch.float64, numel=3 * int(nsteps), optional=True)
        self.ctx.check(_lib.ppmd_md_run_analysed(self.h, int(nsteps), _opt(energies), _opt(qrows),
                                                 1 if use_graph else 0))

    def get_q(self):
        q = torch.empty((3, self.n), dtype=torch.float32, device="cuda")
        self.ctx.check(_lib.ppmd_md_get_q(self.h, _ptr(q[0]), _ptr(q[1]), _ptr(q[2])))
        return q

    def get_state(self, pos=None, vel=None, force=None):
        for t, name in ((pos, "pos"), (vel, "vel"), (force, "force")):
            _need(t, name, torch.float64, (self.n, 3), optional=True)
        self.ctx.check(_lib.ppmd_md_get_state(self.h, _ptr(pos) if pos is not None else None,
                                              _ptr(vel) if vel is not None else None,
                                              _ptr(force) if force is not None else None))

    def forces(self):
        self.ctx.check(_lib.ppmd_md_forces(self.h))

    def list_stats(self):
        pairs, mx = _I64(), _I32()
        self.ctx.check(_lib.ppmd_md_list_stats(self.h, C.byref(pairs), C.byref(mx)))
        return pairs.value, mx.value

    def set_pair_loop(self, mechanism):
        """PAIR_COLUMNS (default) or PAIR_BRICKS; before set_state."""
        self.ctx.check(_lib.ppmd_md_set_pair_loop(self.h, int(mechanism)))

    def set_shape(self, shape):
        """Launch shape k of MD_SHAPES (FP32 atom-index pair loop; 0 is the default)."""
        self.ctx.check(_lib.ppmd_md_set_shape(self.h, int(shape)))

    def get_shape(self):
        """dict(shape, block, per_sm, brick_home) of the present launch shape."""
        v = [_I32() for _ in range(4)]
        self.ctx.check(_lib.ppmd_md_get_shape(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("shape", "block", "per_sm", "brick_home"), (x.value for x in v)))

    def tune(self, steps=20, cache=None):
        """Time every launch shape for `steps` steps from the present state
        (or take the cached choice for this workload) and keep the fastest;
        the state starts again as after set_state.  Returns dict(shape,
        timed, ms_per_step: list (-1 where not timed), and the shape's
        parameters)."""
        shape, timed = _I32(), _I()
        ms = (_D * MD_SHAPES)()
        path = None if cache is None else os.fsencode(cache)
        self.ctx.check(_lib.ppmd_md_tune(self.h, int(steps), path, C.byref(shape), ms, C.byref(timed)))
        out = self.get_shape()
        out.update(timed=bool(timed.value), ms_per_step=[float(x) for x in ms])
        return out

    def set_check(self, on=True):
        """Count, at every later rebuild, pairs within rc that the previous list lacked."""
        self.ctx.check(_lib.ppmd_md_set_check(self.h, 1 if on else 0))

    def missed_pairs(self):
        v = _I64()
        self.ctx.check(_lib.ppmd_md_missed_pairs(self.h, C.byref(v)))
        return v.value

    def time_pair_loops(self, on=True):
        self.ctx.check(_lib.ppmd_md_time_pair_loops(self.h, 1 if on else 0))

    def pair_loop_times(self):
        """(ms per fused pair loop, count, ms per other pair loop, count) of the last replayed graph."""
        a, na, b, nb = _D(), _I32(), _D(), _I32()
        self.ctx.check(_lib.ppmd_md_pair_loop_times(self.h, C.byref(a), C.byref(na), C.byref(b), C.byref(nb)))
        return a.value, na.value, b.value, nb.value

    def get_list(self, max_nbr=None):
        """The last build's list in caller order: (nbr [n, max_nbr] int32 caller indices, count [n])."""
        max_nbr = self.params.max_nbr if max_nbr is None else max_nbr
        nbr = torch.full((self.n, max_nbr), -1, dtype=torch.int32, device="cuda")
        cnt = torch.empty(self.n, dtype=torch.int32, device="cuda")
        self.ctx.check(_lib.ppmd_md_get_list(self.h, _ptr(nbr), _ptr(cnt), int(max_nbr)))
        return nbr, cnt

    def info(self):
        s, r, d = _I64(), _I64(), _D()
        code = _lib.ppmd_md_info(self.h, C.byref(s), C.byref(r), C.byref(d))
        self.ctx.check(code)
        return dict(steps=s.value, rebuilds=r.value, max_disp=d.value, status=code)


NOALLOC_MAX_ATOMS = 262144


def ppmd_lj_forces_noalloc(pos, box, nbr, nbr_count, force, e_atom, totals, rc=2.5, eps=1.0, sigma=1.0, shift=0.0,
                           prec=FP32, stream=None, n=None):
    """ppmd_lj_forces into caller-allocated outputs, with no context and no
    allocation by the library (for callers that may not allocate device
    memory).  totals: float64 CUDA tensor of 2 (U, W) or None.  Returns the
    C status code."""
    if stream is None:
        stream = torch.cuda.current_stream()
    # n differs from the arrays' length only to exercise the size limit (the
    # call refuses it before reading anything)
    if n is None or n <= NOALLOC_MAX_ATOMS:
        n = pos.shape[0]
        if pos.dtype != torch.float64 or tuple(pos.shape) != (n, 3) or not pos.is_contiguous():
            raise ValueError("pos: contiguous float64 [n][3]")
        if force.dtype != torch.float64 or tuple(force.shape) != (n, 3) or not force.is_contiguous():
            raise ValueError("force: contiguous float64 [n][3]")
        if nbr.dtype != torch.int32 or nbr.dim() != 2 or nbr.shape[0] != n or not nbr.is_contiguous():
            raise ValueError("nbr: contiguous int32 [n][max_nbr]")
        if nbr_count.dtype != torch.int32 or tuple(nbr_count.shape) != (n,):
            raise ValueError("nbr_count: int32 [n]")
        if e_atom is not None and (e_atom.dtype != torch.float64 or tuple(e_atom.shape) != (n,)):
            raise ValueError("e_atom: float64 [n]")
        if totals is not None and (totals.dtype != torch.float64 or totals.numel() < 2):
            raise ValueError("totals: float64 [2]")
    p = LJParams(eps, sigma, rc, shift)
    b = _box(box)
    max_nbr = nbr.shape[1] if nbr.dim() == 2 else 0
    return _lib.ppmd_lj_forces_noalloc(C.c_void_p(stream.cuda_stream), _ptr(pos), int(n), C.byref(b), C.byref(p),
                                       _ptr(nbr), _ptr(nbr_count), int(max_nbr), int(prec), _ptr(force),
                                       _ptr(e_atom) if e_atom is not None else None,
                                       _ptr(totals[0:1]) if totals is not None else None,
                                       C.c_void_p(totals.data_ptr() + 8) if totals is not None else None)
