"""Thin ctypes binding of libovs (include/ovs.h): the same entry points, argument marshalling only.

Every computation of the assembly and interpolation path runs in libovs's CUDA kernels.  PyTorch is used
only for device memory and streams.  There is no CPU fallback: if libovs.so is missing or no GPU is
present, these functions raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libovs.so")

OVS_OK = 0
OVS_ERR_ARG = -1
OVS_ERR_STATE = -2
OVS_ERR_WORKSPACE = -3
OVS_ERR_CUDA = -4
OVS_ERR_NO_DEVICE = -5
OVS_ERR_DEVICE = -6

OVS_STATUS_FOUND = 0
OVS_STATUS_ORPHAN = 1
OVS_STATUS_BADINPUT = 2
OVS_STATUS_MASK = 0x0F
OVS_STATUS_FALLBACK = 0x10
OVS_STATUS_REFINED = 0x20

OVS_F32 = 0
OVS_F64 = 1

OVS_MAX_GRIDS = 31
OVS_MAX_SETS = 64
OVS_MAX_DONORS = 8

OVS_VEL_RELATIVE = 0
OVS_VEL_ABSOLUTE = 1
OVS_VEL_NONE = 2

OVS_GUESS_HINT = 0
OVS_GUESS_BINS = 1
OVS_GUESS_MLP = 2
OVS_GUESS_MLP_ONLY = 3
OVS_LAUNCH_DIRECT = 0
OVS_LAUNCH_GRAPH = 1

EXPORTS = [
    "ovs_ctx_create", "ovs_ctx_destroy", "ovs_last_error", "ovs_set_stream", "ovs_workspace_size",
    "ovs_workspace_attach", "ovs_grid_workspace_size", "ovs_create_grid", "ovs_set_motion", "ovs_set_options",
    "ovs_get_options", "ovs_assemble", "ovs_interpolate", "ovs_sync", "ovs_get_stats", "ovs_reset_hints",
    "ovs_set_trace_events", "ovs_assemble_noalloc", "ovs_assemble_interpolate", "ovs_guess_param_count",
    "ovs_train_workspace_size", "ovs_train_guess", "ovs_guess_get_params", "ovs_guess_set_params",
    "ovs_guess_eval", "ovs_mlp_loss_grad", "ovs_set_tuning", "ovs_get_tuning", "ovs_autotune",
    "ovs_interp_matrix", "ovs_spmv", "ovs_set_iblank", "ovs_surface_workspace_size", "ovs_create_surface",
    "ovs_hole_cut",
    "ovs_hole_cut_many",
    "ovs_get_donors",
    "ovs_set_donors",
    "ovs_autotune_guess",
    "ovs_interface_flux",
    "ovs_grid_check",
    "ovs_set_grid_overlap",
    "ovs_grid_bins",
]

OVS_NOALLOC_MAX_POINTS = 1 << 20


class ovs_grid_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("periodic", ctypes.c_int32 * 3), ("x", ctypes.c_void_p),
                ("y", ctypes.c_void_p), ("z", ctypes.c_void_p), ("role", ctypes.c_int32)]


class ovs_fringe_set(ctypes.Structure):
    _fields_ = [("receiver", ctypes.c_int32), ("n_donors", ctypes.c_int32),
                ("donors", ctypes.c_int32 * OVS_MAX_DONORS), ("n", ctypes.c_int64), ("node_ids", ctypes.c_void_p)]


class ovs_donors(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("grid", ctypes.c_void_p), ("cell", ctypes.c_void_p), ("xi", ctypes.c_void_p),
                ("xi_dtype", ctypes.c_int32), ("status", ctypes.c_void_p)]


class ovs_fields(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("dtype", ctypes.c_int32), ("stride", ctypes.c_int32)]


class ovs_fields_out(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("dtype", ctypes.c_int32)]


class ovs_options(ctypes.Structure):
    _fields_ = [("velocity_mode", ctypes.c_int32), ("guess", ctypes.c_int32), ("max_walk", ctypes.c_int32),
                ("collect_stats", ctypes.c_int32), ("launch", ctypes.c_int32)]


class ovs_tuning(ctypes.Structure):
    _fields_ = [("assemble_blocks_per_sm", ctypes.c_int32), ("interp_blocks_per_sm", ctypes.c_int32),
                ("slow_blocks_per_sm", ctypes.c_int32), ("guess_blocks_per_sm", ctypes.c_int32),
                ("launch", ctypes.c_int32)]


class ovs_stats(ctypes.Structure):
    _fields_ = [("points", ctypes.c_int64), ("walk_steps", ctypes.c_int64), ("refined", ctypes.c_int64),
                ("fallback", ctypes.c_int64), ("guess_used", ctypes.c_int64), ("newton_iterations", ctypes.c_int64),
                ("warp_walk_steps", ctypes.c_int64), ("near_face", ctypes.c_int64), ("stuck", ctypes.c_int64)]


class ovs_train_desc(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int32), ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("lr", ctypes.c_float), ("lr_final", ctypes.c_float), ("pad", ctypes.c_int32),
                ("n_samples", ctypes.c_int64), ("cells", ctypes.c_void_p),
                ("xi", ctypes.c_void_p), ("init_params", ctypes.c_void_p), ("scratch", ctypes.c_void_p),
                ("scratch_bytes", ctypes.c_size_t)]


class OvsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libovs error {code}: {msg}")
        self.code = code


_lib = None


def load(path: Optional[str] = None):
    """Load libovs.so (built by ``paper_1910_09315_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libovs.so not built ({p}); run paper_1910_09315_gb300/build.py")
    L = ctypes.CDLL(p)
    V, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "ovs_ctx_create": [ctypes.POINTER(V), ctypes.c_int, V],
        "ovs_ctx_destroy": [V],
        "ovs_last_error": [V],
        "ovs_set_stream": [V, V],
        "ovs_workspace_size": [V, I64, ctypes.POINTER(SZ)],
        "ovs_workspace_attach": [V, V, SZ, I64],
        "ovs_grid_workspace_size": [ctypes.POINTER(ovs_grid_desc), ctypes.POINTER(SZ)],
        "ovs_create_grid": [V, ctypes.POINTER(ovs_grid_desc), V, SZ, ctypes.POINTER(I32)],
        "ovs_set_motion": [V, I32, V, V, V, V],
        "ovs_set_options": [V, ctypes.POINTER(ovs_options)],
        "ovs_get_options": [V, ctypes.POINTER(ovs_options)],
        "ovs_assemble": [V, ctypes.POINTER(ovs_fringe_set), I32, ctypes.POINTER(ovs_donors)],
        "ovs_interpolate": [V, ctypes.POINTER(ovs_fringe_set), I32, ctypes.POINTER(ovs_donors),
                            ctypes.POINTER(ovs_fields), I32, ctypes.POINTER(ovs_fields_out)],
        "ovs_sync": [V],
        "ovs_get_stats": [V, ctypes.POINTER(ovs_stats), ctypes.c_int],
        "ovs_reset_hints": [V],
        "ovs_set_trace_events": [V, ctypes.POINTER(V), I32],
        "ovs_assemble_noalloc": [V, ctypes.POINTER(ovs_fringe_set), I32, ctypes.POINTER(ovs_donors)],
        "ovs_assemble_interpolate": [V, ctypes.POINTER(ovs_fringe_set), I32, ctypes.POINTER(ovs_donors),
                                     ctypes.POINTER(ovs_fields), I32, ctypes.POINTER(ovs_fields_out)],
        "ovs_guess_param_count": [I32, ctypes.POINTER(I64)],
        "ovs_train_workspace_size": [ctypes.POINTER(ovs_train_desc), ctypes.POINTER(SZ)],
        "ovs_train_guess": [V, I32, ctypes.POINTER(ovs_train_desc), ctypes.POINTER(ctypes.c_float)],
        "ovs_guess_get_params": [V, I32, V, ctypes.POINTER(I32)],
        "ovs_guess_set_params": [V, I32, I32, V],
        "ovs_guess_eval": [V, I32, I64, V, V],
        "ovs_mlp_loss_grad": [V, I32, I64, V, V, V, V, V],
        "ovs_interp_matrix": [V, ctypes.POINTER(ovs_donors), V, V, V, I32],
        "ovs_set_iblank": [V, I32, V],
        "ovs_surface_workspace_size": [I64, V, I64, V, ctypes.POINTER(SZ)],
        "ovs_create_surface": [V, I32, I64, V, I64, V, V, SZ, ctypes.POINTER(I32)],
        "ovs_hole_cut": [V, I32, I32, I64, V, V],
        "ovs_hole_cut_many": [V, I32, V, I32, V, V, V],
        "ovs_get_donors": [V, I32, V],
        "ovs_set_donors": [V, I32, V],
        "ovs_spmv": [V, I64, V, V, V, V, V, I32],
        "ovs_set_tuning": [V, ctypes.POINTER(ovs_tuning)],
        "ovs_get_tuning": [V, ctypes.POINTER(ovs_tuning)],
        "ovs_autotune": [V, ctypes.POINTER(ovs_fringe_set), I32, ctypes.POINTER(ovs_donors), ctypes.POINTER(ovs_fields),
                         I32, ctypes.POINTER(ovs_fields_out), I32, ctypes.POINTER(ovs_tuning)],
        "ovs_grid_check": [V, I32, V, ctypes.POINTER(I32)],
        "ovs_set_grid_overlap": [V, I32, I32],
        "ovs_grid_bins": [V, I32, V],
        "ovs_interface_flux": [V, I32, I64, V, V, I32, V, ctypes.POINTER(ovs_fields), V, V, I32],
        "ovs_autotune_guess": [V, ctypes.POINTER(ovs_fringe_set), I32, ctypes.POINTER(ovs_donors),
                               ctypes.POINTER(ovs_fields), I32, ctypes.POINTER(ovs_fields_out), I32, V, V, I32, V,
                               ctypes.POINTER(I32)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "ovs_last_error" else ctypes.c_int
    if path is None:
        _lib = L
    return L


def _check(ctx, rc: int):
    if rc != OVS_OK:
        msg = load().ovs_last_error(ctx).decode() if ctx else ""
        raise OvsError(rc, msg)


# ------------------------------------------------------------------ entry points (same names as the C ABI)
def ovs_ctx_create(device: int = 0, stream=None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    rc = load().ovs_ctx_create(ctypes.byref(ctx), int(device), ctypes.c_void_p(_stream_handle(stream)))
    if rc != OVS_OK:
        raise OvsError(rc, "ovs_ctx_create failed (no usable CUDA device?)")
    return ctx


def ovs_ctx_destroy(ctx):
    _check(ctx, load().ovs_ctx_destroy(ctx))


def ovs_last_error(ctx) -> str:
    return load().ovs_last_error(ctx).decode()


def ovs_set_stream(ctx, stream):
    _check(ctx, load().ovs_set_stream(ctx, ctypes.c_void_p(_stream_handle(stream))))


def ovs_workspace_size(ctx, max_points: int) -> int:
    b = ctypes.c_size_t()
    _check(ctx, load().ovs_workspace_size(ctx, int(max_points), ctypes.byref(b)))
    return b.value


def ovs_workspace_attach(ctx, dptr: int, nbytes: int, max_points: int):
    _check(ctx, load().ovs_workspace_attach(ctx, ctypes.c_void_p(dptr), nbytes, int(max_points)))


def ovs_grid_workspace_size(desc: ovs_grid_desc) -> int:
    b = ctypes.c_size_t()
    rc = load().ovs_grid_workspace_size(ctypes.byref(desc), ctypes.byref(b))
    if rc != OVS_OK:
        raise OvsError(rc, "invalid grid descriptor")
    return b.value


def ovs_create_grid(ctx, desc: ovs_grid_desc, dptr: int, nbytes: int) -> int:
    gid = ctypes.c_int32()
    _check(ctx, load().ovs_create_grid(ctx, ctypes.byref(desc), ctypes.c_void_p(dptr), nbytes, ctypes.byref(gid)))
    return gid.value


def ovs_set_motion(ctx, grid_id: int, R, c, V, omega):
    arrs = [(ctypes.c_double * n)(*[float(x) for x in a]) for a, n in ((_flat(R), 9), (_flat(c), 3), (_flat(V), 3),
                                                                       (_flat(omega), 3))]
    _check(ctx, load().ovs_set_motion(ctx, int(grid_id), *[ctypes.cast(a, ctypes.c_void_p) for a in arrs]))


def ovs_set_options(ctx, opts: ovs_options):
    _check(ctx, load().ovs_set_options(ctx, ctypes.byref(opts)))


def ovs_get_options(ctx) -> ovs_options:
    o = ovs_options()
    _check(ctx, load().ovs_get_options(ctx, ctypes.byref(o)))
    return o


def ovs_assemble(ctx, sets, nsets: int, donors: ovs_donors):
    _check(ctx, load().ovs_assemble(ctx, sets, int(nsets), ctypes.byref(donors)))


def ovs_assemble_interpolate(ctx, sets, nsets: int, donors: ovs_donors, fields, nfields: int, out: ovs_fields_out):
    _check(ctx, load().ovs_assemble_interpolate(ctx, sets, int(nsets), ctypes.byref(donors), fields, int(nfields),
                                                ctypes.byref(out)))


def ovs_set_iblank(ctx, grid_id: int, iblank: int):
    """iblank: device pointer to uint8 [nodes] (0 = blanked), or 0 / None for every node active."""
    _check(ctx, load().ovs_set_iblank(ctx, int(grid_id), iblank or None))


def ovs_surface_workspace_size(V, T) -> int:
    """V: float64 (nv, 3) host vertices, T: int32 (nt, 3) host triangles."""
    import numpy as np

    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    out = ctypes.c_size_t(0)
    rc = load().ovs_surface_workspace_size(len(V), V.ctypes.data, len(T), T.ctypes.data, ctypes.byref(out))
    if rc != OVS_OK:
        raise OvsError(rc, "ovs_surface_workspace_size: bad surface")
    return out.value


def ovs_create_surface(ctx, body_grid: int, V, T, dws: int, nbytes: int) -> int:
    import numpy as np

    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    sid = ctypes.c_int32(0)
    _check(ctx, load().ovs_create_surface(ctx, int(body_grid), len(V), V.ctypes.data, len(T), T.ctypes.data, dws,
                                          int(nbytes), ctypes.byref(sid)))
    return sid.value


def ovs_hole_cut(ctx, surface_id: int, target_grid: int, n: int, nodes: int, iblank: int):
    _check(ctx, load().ovs_hole_cut(ctx, int(surface_id), int(target_grid), int(n), nodes or None, iblank))


def ovs_hole_cut_many(ctx, surface_ids, target_grid: int, ns, nodes, iblank: int):
    """surface_ids, ns: sequences of ints; nodes: sequence of device pointers (int, or None for 0 .. n-1)."""
    k = len(surface_ids)
    ids = (ctypes.c_int32 * max(1, k))(*[int(x) for x in surface_ids])
    nn = (ctypes.c_int64 * max(1, k))(*[int(x) for x in ns])
    nd = (ctypes.c_void_p * max(1, k))(*[(p or None) for p in nodes])
    _check(ctx, load().ovs_hole_cut_many(ctx, k, ids, int(target_grid), nn, nd, iblank))


def ovs_interp_matrix(ctx, donors: ovs_donors, row_ptr: int, col: int, val: int, val_dtype: int):
    _check(ctx, load().ovs_interp_matrix(ctx, ctypes.byref(donors), row_ptr, col, val, int(val_dtype)))


def ovs_spmv(ctx, nrows: int, row_ptr: int, col: int, val: int, x: int, y: int, dtype: int):
    _check(ctx, load().ovs_spmv(ctx, int(nrows), row_ptr, col, val, x, y, int(dtype)))


def ovs_set_tuning(ctx, t):
    """t: ovs_tuning or None (defaults)."""
    _check(ctx, load().ovs_set_tuning(ctx, ctypes.byref(t) if t is not None else None))


def ovs_get_tuning(ctx) -> ovs_tuning:
    t = ovs_tuning()
    _check(ctx, load().ovs_get_tuning(ctx, ctypes.byref(t)))
    return t


def ovs_autotune(ctx, sets, nsets: int, donors: ovs_donors, fields, nfields: int, out, reps: int) -> ovs_tuning:
    """out: ovs_fields_out or None (tune ovs_assemble alone)."""
    best = ovs_tuning()
    _check(ctx, load().ovs_autotune(ctx, sets, int(nsets), ctypes.byref(donors), fields, int(nfields),
                                    ctypes.byref(out) if out is not None else None, int(reps), ctypes.byref(best)))
    return best


def ovs_autotune_guess(ctx, sets, nsets: int, donors: ovs_donors, fields, nfields: int, out, hidden, params,
                       reps: int):
    """hidden: candidate widths (0 = no networks); params: per candidate a list over grids of device parameter
    pointers (int, 0 for none).  Returns (best index, [(cold ms, warm ms) per candidate])."""
    nc = len(hidden)
    ng = len(params[0]) if params else 0
    h = (ctypes.c_int32 * nc)(*[int(x) for x in hidden])
    flat = [int(p) for cand in params for p in cand]
    parr = (ctypes.c_void_p * max(1, len(flat)))(*[p or None for p in flat]) if flat else None
    ms = (ctypes.c_float * (2 * nc))()
    best = ctypes.c_int32()
    assert not flat or len(flat) == nc * ng
    _check(ctx, load().ovs_autotune_guess(ctx, sets, int(nsets), ctypes.byref(donors), fields, int(nfields),
                                          ctypes.byref(out) if out is not None else None, nc, h, parr, int(reps), ms,
                                          ctypes.byref(best)))
    return best.value, [(ms[2 * k], ms[2 * k + 1]) for k in range(nc)]


def ovs_interface_flux(ctx, grid_id: int, nfaces: int, faces: int, signs: int, nsurf: int, surf_start, vel: ovs_fields,
                       flux: int, net: int, correct: bool):
    """Pointers as ints (device), surf_start a host sequence of nsurf + 1 offsets."""
    ss = (ctypes.c_int64 * max(1, nsurf + 1))(*[int(x) for x in (surf_start if nsurf else [0])])
    _check(ctx, load().ovs_interface_flux(ctx, int(grid_id), int(nfaces), ctypes.c_void_p(faces or None),
                                          ctypes.c_void_p(signs or None), int(nsurf), ss if nsurf else None,
                                          ctypes.byref(vel), ctypes.c_void_p(flux or None),
                                          ctypes.c_void_p(net or None), int(bool(correct))))


def ovs_grid_check(ctx, grid_id: int):
    """(cells right-handed, left-handed, folded or degenerate), and whether the grid is searched exhaustively."""
    cells = (ctypes.c_int64 * 3)()
    ov = ctypes.c_int32()
    _check(ctx, load().ovs_grid_check(ctx, int(grid_id), cells, ctypes.byref(ov)))
    return tuple(int(x) for x in cells), bool(ov.value)


def ovs_grid_bins(ctx, grid_id: int):
    """(control cells, their registrations, crowded control cells split into finer bins, finer-bin registrations)."""
    out = (ctypes.c_int64 * 4)()
    _check(ctx, load().ovs_grid_bins(ctx, int(grid_id), out))
    return tuple(int(x) for x in out)


def ovs_set_grid_overlap(ctx, grid_id: int, overlap: bool):
    _check(ctx, load().ovs_set_grid_overlap(ctx, int(grid_id), int(bool(overlap))))


def ovs_assemble_noalloc(ctx, sets, nsets: int, donors: ovs_donors):
    """ovs_assemble with its slow-path queue in the library's fixed device array: allocates nothing, at most
    OVS_NOALLOC_MAX_POINTS points per call (see include/ovs.h)."""
    _check(ctx, load().ovs_assemble_noalloc(ctx, sets, int(nsets), ctypes.byref(donors)))


def ovs_interpolate(ctx, sets, nsets: int, donors: ovs_donors, fields, nfields: int, out: ovs_fields_out):
    _check(ctx, load().ovs_interpolate(ctx, sets, int(nsets), ctypes.byref(donors), fields, int(nfields),
                                       ctypes.byref(out)))


def ovs_guess_param_count(hidden: int) -> int:
    n = ctypes.c_int64()
    rc = load().ovs_guess_param_count(int(hidden), ctypes.byref(n))
    if rc != OVS_OK:
        raise OvsError(rc, f"hidden width {hidden}")
    return n.value


def ovs_train_workspace_size(desc: ovs_train_desc) -> int:
    b = ctypes.c_size_t()
    rc = load().ovs_train_workspace_size(ctypes.byref(desc), ctypes.byref(b))
    if rc != OVS_OK:
        raise OvsError(rc, "invalid training descriptor")
    return b.value


def ovs_train_guess(ctx, grid_id: int, desc: ovs_train_desc) -> float:
    loss = ctypes.c_float()
    _check(ctx, load().ovs_train_guess(ctx, int(grid_id), ctypes.byref(desc), ctypes.byref(loss)))
    return loss.value


def ovs_guess_get_params(ctx, grid_id: int, dptr: int) -> int:
    h = ctypes.c_int32()
    _check(ctx, load().ovs_guess_get_params(ctx, int(grid_id), ctypes.c_void_p(dptr), ctypes.byref(h)))
    return h.value


def ovs_guess_set_params(ctx, grid_id: int, hidden: int, dptr: int):
    _check(ctx, load().ovs_guess_set_params(ctx, int(grid_id), int(hidden), ctypes.c_void_p(dptr)))


def ovs_guess_eval(ctx, grid_id: int, n: int, xn_ptr: int, out_ptr: int):
    _check(ctx, load().ovs_guess_eval(ctx, int(grid_id), int(n), ctypes.c_void_p(xn_ptr), ctypes.c_void_p(out_ptr)))


def ovs_mlp_loss_grad(ctx, hidden: int, n: int, xn_ptr: int, t_ptr: int, params_ptr: int, grads_ptr: int,
                      loss_ptr: int):
    _check(ctx, load().ovs_mlp_loss_grad(ctx, int(hidden), int(n), *[ctypes.c_void_p(p) for p in
                                                                      (xn_ptr, t_ptr, params_ptr, grads_ptr,
                                                                       loss_ptr)]))


def ovs_sync(ctx):
    _check(ctx, load().ovs_sync(ctx))


def ovs_get_stats(ctx, reset: bool = False) -> dict:
    s = ovs_stats()
    _check(ctx, load().ovs_get_stats(ctx, ctypes.byref(s), int(bool(reset))))
    return {k: getattr(s, k) for k, _ in ovs_stats._fields_}


def ovs_reset_hints(ctx):
    _check(ctx, load().ovs_reset_hints(ctx))


def ovs_get_donors(ctx, grid_id: int, dst: int):
    """dst: device pointer to uint32 [the grid's node count]."""
    _check(ctx, load().ovs_get_donors(ctx, int(grid_id), dst))


def ovs_set_donors(ctx, grid_id: int, src: int):
    """src: device pointer to uint32 [the grid's node count]."""
    _check(ctx, load().ovs_set_donors(ctx, int(grid_id), src))


def ovs_set_trace_events(ctx, events):
    """events: sequence of torch.cuda.Event (or None) -> recorded at the points include/ovs.h lists.  A torch
    event exists only after its first record(), so record each once before passing it."""
    n = len(events)
    arr = (ctypes.c_void_p * max(1, n))()
    for i, e in enumerate(events):
        if e is not None and not int(e.cuda_event):
            raise ValueError("torch.cuda.Event has no CUDA event yet: record() it once first")
        arr[i] = None if e is None else int(e.cuda_event)
    _check(ctx, load().ovs_set_trace_events(ctx, arr, n))


# ------------------------------------------------------------------ marshalling helpers
def _flat(a) -> List[float]:
    try:
        import numpy as np

        return list(np.asarray(a, dtype=float).reshape(-1))
    except Exception:  # pragma: no cover
        return [float(x) for x in a]


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def make_sets(sets: Sequence) -> "ctypes.Array":
    """sets: sequence of (receiver, node_ids torch int32 cuda tensor, donors list)."""
    arr = (ovs_fringe_set * max(1, len(sets)))()
    for i, (rec, ids, donors) in enumerate(sets):
        arr[i].receiver = int(rec)
        arr[i].n_donors = len(donors)
        for j, d in enumerate(donors):
            arr[i].donors[j] = int(d)
        arr[i].n = int(ids.numel())
        arr[i].node_ids = ids.data_ptr() if ids.numel() else None
    return arr


class Context:
    """Owns an ovs context and the device workspaces it needs (allocated as torch tensors)."""

    def __init__(self, device: int = 0, stream=None, max_points: int = 1 << 20):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libovs needs a CUDA device; there is no CPU fallback")
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = ovs_ctx_create(device, self.stream)
        self.max_points = int(max_points)
        nbytes = ovs_workspace_size(self.ctx, self.max_points)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ovs_workspace_attach(self.ctx, _aligned(self._ws), nbytes, self.max_points)
        self.grids = []  # (desc, coords tensors, workspace)

    def close(self):
        if self.ctx:
            ovs_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_grid(self, x, y, z, dims, periodic=(False, False, False), role: int = 1) -> int:
        t = self.torch
        xs = [a if isinstance(a, t.Tensor) else t.as_tensor(a) for a in (x, y, z)]
        xs = [a.to(device=self.device, dtype=t.float64).contiguous() for a in xs]
        d = ovs_grid_desc()
        for a in range(3):
            d.n[a] = int(dims[a])
            d.periodic[a] = int(bool(periodic[a]))
        d.x, d.y, d.z = xs[0].data_ptr(), xs[1].data_ptr(), xs[2].data_ptr()
        d.role = int(role)
        nbytes = ovs_grid_workspace_size(d)
        ws = t.empty(nbytes + 256, dtype=t.uint8, device=self.device)
        gid = ovs_create_grid(self.ctx, d, _aligned(ws), nbytes)
        self.grids.append((d, xs, ws))
        return gid

    def set_motion(self, gid: int, R, c, V, omega):
        ovs_set_motion(self.ctx, gid, R, c, V, omega)

    def set_options(self, **kw):
        o = ovs_get_options(self.ctx)
        for k, v in kw.items():
            setattr(o, k, int(v))
        ovs_set_options(self.ctx, o)

    def alloc_donors(self, n: int, xi_dtype: int = OVS_F32):
        t = self.torch
        dt = t.float64 if xi_dtype == OVS_F64 else t.float32
        return {"grid": t.empty(n, dtype=t.int32, device=self.device),
                "cell": t.empty(n, dtype=t.int32, device=self.device),
                "xi": t.empty(3 * n, dtype=dt, device=self.device),
                "status": t.empty(n, dtype=t.uint8, device=self.device), "xi_dtype": xi_dtype, "n": n}

    @staticmethod
    def donors_struct(d) -> ovs_donors:
        s = ovs_donors()
        s.n = d["n"]
        s.grid, s.cell, s.xi, s.status = (d["grid"].data_ptr(), d["cell"].data_ptr(), d["xi"].data_ptr(),
                                          d["status"].data_ptr())
        s.xi_dtype = d["xi_dtype"]
        return s

    def assemble(self, sets, donors=None, xi_dtype: int = OVS_F32):
        n = sum(int(s[1].numel()) for s in sets)
        if donors is None:
            donors = self.alloc_donors(n, xi_dtype)
        arr = make_sets(sets)
        ovs_assemble(self.ctx, arr, len(sets), self.donors_struct(donors))
        return donors

    def interpolate(self, sets, donors, fields, out=None):
        """fields: list indexed by grid id of (u, v, w, p) cuda tensors (or None)."""
        farr, o, out = self._fields_structs(fields, donors["n"], out)
        ovs_interpolate(self.ctx, make_sets(sets), len(sets), self.donors_struct(donors), farr, len(self.grids), o)
        return out

    def _fields_structs(self, fields, n, out):
        """fields[g]: (u, v, w, p) tensors, or one (nodes, k >= 4) tensor whose rows hold (u, v, w, p, ...) (rows
        evenly spaced, columns contiguous: the row spacing is the stride)."""
        t = self.torch
        dtype = None
        farr = (ovs_fields * len(self.grids))()
        for g, f in enumerate(fields):
            if f is None:
                continue
            if isinstance(f, t.Tensor):
                assert f.dim() == 2 and f.shape[1] >= 4 and f.stride(1) == 1
                base, es = f.data_ptr(), f.element_size()
                farr[g].u, farr[g].v, farr[g].w, farr[g].p = (base + c * es for c in range(4))
                farr[g].stride = f.stride(0)
                dt = f.dtype
            else:
                farr[g].u, farr[g].v, farr[g].w, farr[g].p = (a.data_ptr() for a in f)
                dt = f[0].dtype
            farr[g].dtype = OVS_F64 if dt == t.float64 else OVS_F32
            dtype = dt
        if out is None:
            out = [t.empty(n, dtype=dtype, device=self.device) for _ in range(4)]
        o = ovs_fields_out()
        o.u, o.v, o.w, o.p = (a.data_ptr() for a in out)
        o.dtype = OVS_F64 if out[0].dtype == t.float64 else OVS_F32
        return farr, o, out

    def assemble_interpolate(self, sets, fields, donors=None, out=None, xi_dtype: int = OVS_F32):
        """ovs_assemble_interpolate: donors and interpolated fields in one call."""
        n = sum(int(s[1].numel()) for s in sets)
        if donors is None:
            donors = self.alloc_donors(n, xi_dtype)
        farr, o, out = self._fields_structs(fields, n, out)
        ovs_assemble_interpolate(self.ctx, make_sets(sets), len(sets), self.donors_struct(donors), farr,
                                 len(self.grids), o)
        return donors, out

    def autotune(self, sets, fields=None, donors=None, out=None, reps: int = 5, xi_dtype: int = OVS_F32) -> dict:
        """ovs_autotune on this call (with interpolation when fields are given); returns the chosen shapes."""
        n = sum(int(s[1].numel()) for s in sets)
        if donors is None:
            donors = self.alloc_donors(n, xi_dtype)
        if fields is not None:
            farr, o, out = self._fields_structs(fields, n, out)
            best = ovs_autotune(self.ctx, make_sets(sets), len(sets), self.donors_struct(donors), farr,
                                len(self.grids), o, reps)
        else:
            best = ovs_autotune(self.ctx, make_sets(sets), len(sets), self.donors_struct(donors), None, 0, None, reps)
        return {k: getattr(best, k) for k, _ in ovs_tuning._fields_}

    def autotune_guess(self, sets, fields, hidden, params, donors=None, out=None, reps: int = 3,
                       xi_dtype: int = OVS_F32):
        """ovs_autotune_guess on this call: hidden = candidate widths (0 = no networks), params[k][g] = a device
        FP32 parameter tensor of grid g for candidate k (or None).  Returns (chosen index, [(cold ms, warm ms)])."""
        n = sum(int(s[1].numel()) for s in sets)
        if donors is None:
            donors = self.alloc_donors(n, xi_dtype)
        ptrs = [[(p.data_ptr() if p is not None else 0) for p in cand] for cand in params]
        if fields is not None:
            farr, o, out = self._fields_structs(fields, n, out)
            return ovs_autotune_guess(self.ctx, make_sets(sets), len(sets), self.donors_struct(donors), farr,
                                      len(self.grids), o, hidden, ptrs, reps)
        return ovs_autotune_guess(self.ctx, make_sets(sets), len(sets), self.donors_struct(donors), None, 0, None,
                                  hidden, ptrs, reps)

    def interface_flux(self, gid: int, faces, vel, signs=None, surf_start=None, correct: bool = False):
        """ovs_interface_flux: faces device int64 tensor, vel = (u, v, w) device tensors over grid gid's nodes,
        signs device int8 tensor or None, surf_start host list (nsurf + 1) or None.  Returns (flux, net) where net
        is a device FP64 tensor [2 nsurf] (net flux before the correction, total area) or None."""
        t = self.torch
        nsurf = 0 if surf_start is None else len(surf_start) - 1
        flux = t.empty(int(faces.numel()), dtype=vel[0].dtype, device=self.device)
        net = t.empty(max(1, 2 * nsurf), dtype=t.float64, device=self.device) if nsurf else None
        v = ovs_fields()
        v.u, v.v, v.w, v.p = vel[0].data_ptr(), vel[1].data_ptr(), vel[2].data_ptr(), vel[0].data_ptr()
        v.dtype = OVS_F64 if vel[0].dtype == t.float64 else OVS_F32
        v.stride = 1
        ovs_interface_flux(self.ctx, gid, int(faces.numel()), faces.data_ptr(),
                           signs.data_ptr() if signs is not None else 0, nsurf, surf_start, v, flux.data_ptr(),
                           net.data_ptr() if net is not None else 0, correct)
        return flux, net

    def add_surface(self, body_gid: int, V, T) -> int:
        """ovs_create_surface of a closed triangulated body surface (host V (nv, 3), T (nt, 3)) fixed in grid
        body_gid's frame; the workspace is a torch tensor kept alive by this context."""
        nbytes = ovs_surface_workspace_size(V, T)
        ws = self.torch.empty(nbytes + 256, dtype=self.torch.uint8, device=self.device)
        ptr = _aligned(ws)
        sid = ovs_create_surface(self.ctx, body_gid, V, T, ptr, nbytes)
        self._surface_ws = getattr(self, "_surface_ws", []) + [ws]
        return sid

    def hole_cut(self, sid: int, target_gid: int, iblank, nodes=None):
        """ovs_hole_cut: zero iblank (device uint8 tensor over target_gid's nodes) at the given nodes (device
        int32 tensor, or None for all nodes) that lie inside surface sid."""
        n = int(nodes.numel()) if nodes is not None else int(iblank.numel())
        ovs_hole_cut(self.ctx, sid, target_gid, n, nodes.data_ptr() if nodes is not None else None,
                     iblank.data_ptr())

    def get_donors(self, gid: int):
        """ovs_get_donors: grid gid's previous donors as a device int32 tensor (the uint32 bits), one per node."""
        d = self.grids[gid][0]
        out = self.torch.empty(int(d.n[0]) * int(d.n[1]) * int(d.n[2]), dtype=self.torch.int32, device=self.device)
        ovs_get_donors(self.ctx, gid, out.data_ptr())
        return out

    def set_donors(self, gid: int, donors):
        """ovs_set_donors from a device int32 tensor of get_donors' layout (kept alive by this context until the
        copy has run: the caller synchronises or keeps the tensor)."""
        assert donors.dtype == self.torch.int32 and donors.is_contiguous()
        ovs_set_donors(self.ctx, gid, donors.data_ptr())

    def hole_cut_many(self, sids, target_gid: int, iblank, nodes):
        """ovs_hole_cut_many: surfaces sids cut iblank in one launch; nodes: one device int32 tensor per surface
        (or None for all of the target grid's nodes)."""
        ns = [int(x.numel()) if x is not None else int(iblank.numel()) for x in nodes]
        ptrs = [x.data_ptr() if x is not None else None for x in nodes]
        ovs_hole_cut_many(self.ctx, list(sids), target_gid, ns, ptrs, iblank.data_ptr())

    def interp_matrix(self, donors, val_dtype: int = OVS_F32):
        """ovs_interp_matrix of a donors dict -> (row_ptr int32 [n+1], col int64 [8n], val [8n]) on the device."""
        t = self.torch
        n = donors["n"]
        row_ptr = t.empty(n + 1, dtype=t.int32, device=self.device)
        col = t.empty(max(1, 8 * n), dtype=t.int64, device=self.device)
        val = t.empty(max(1, 8 * n), dtype=t.float64 if val_dtype == OVS_F64 else t.float32, device=self.device)
        ovs_interp_matrix(self.ctx, self.donors_struct(donors), row_ptr.data_ptr(), col.data_ptr(), val.data_ptr(),
                          val_dtype)
        return row_ptr, col, val

    def spmv(self, row_ptr, col, val, x):
        """y = A x (ovs_spmv); x: device vector of all grids' node values in the global numbering."""
        t = self.torch
        nrows = int(row_ptr.numel()) - 1
        y = t.empty(max(1, nrows), dtype=val.dtype, device=self.device)
        ovs_spmv(self.ctx, nrows, row_ptr.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr(), y.data_ptr(),
                 OVS_F64 if val.dtype == t.float64 else OVS_F32)
        return y[:nrows]

    def set_tuning(self, **kw):
        t = ovs_get_tuning(self.ctx)
        for k, v in kw.items():
            setattr(t, k, int(v))
        ovs_set_tuning(self.ctx, t)

    def train_guess(self, gid: int, cells, xi, init_params, hidden: int = 64, epochs: int = 5, batch: int = 8192,
                    lr: float = 3e-3, lr_final: float = 0.0) -> float:
        """Train grid gid's guess network (cells int32 [n], xi float32 [n,3] or [3n] SoA, init_params float32)."""
        t = self.torch
        cells = t.as_tensor(cells, dtype=t.int32).to(self.device).contiguous()
        xi = t.as_tensor(xi, dtype=t.float32).to(self.device)
        if xi.dim() == 2:
            xi = xi.t().contiguous().reshape(-1)
        init = t.as_tensor(init_params, dtype=t.float32).to(self.device).contiguous()
        d = ovs_train_desc()
        d.hidden, d.epochs, d.batch, d.lr, d.lr_final = int(hidden), int(epochs), int(batch), float(lr), float(lr_final)
        d.n_samples = int(cells.numel())
        d.cells, d.xi, d.init_params = cells.data_ptr(), xi.data_ptr(), init.data_ptr()
        nbytes = ovs_train_workspace_size(d)
        scratch = t.empty(nbytes, dtype=t.uint8, device=self.device)
        d.scratch, d.scratch_bytes = scratch.data_ptr(), nbytes
        return ovs_train_guess(self.ctx, gid, d)

    def sync(self):
        ovs_sync(self.ctx)

    def stats(self, reset=False):
        return ovs_get_stats(self.ctx, reset)


def _aligned(t) -> int:
    p = t.data_ptr()
    return (p + 255) // 256 * 256
