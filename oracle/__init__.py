"""Plain FP64 CPU oracle for the overset assembly + interpolation path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.

Parts (each cites the passage it follows):

* ``ovs_oracle.c`` -- cells, trilinear shape functions, FP64 Newton in-cell
  predicate, control-cell bins, lowest-id selection (Sec. 2.2.5 donor search,
  Algorithm "donor search", Sec. 2.2.6 trilinear interpolation).
* ``frame_map`` -- receiver frame -> inertial -> donor frame (Sec. 2.1,
  eq. "velocity" and Fig. "non-inertial": x_in = R x_body + c).
* ``assemble`` -- donor selection over a priority list of donor grids
  (Sec. 2.4 item 1: the first grid in the list that has a donor wins).
* ``interpolate`` -- q = sum_a N_a(xi) q_a (Sec. 2.2.6) and the frame
  velocity transform: RELATIVE  u_in = R_d u_d + V_d + omega_d x (x_in - c_d),
  u_r = R_r^T (u_in - V_r - omega_r x (x_in - c_r)) (Sec. 2.1 eq. "velocity":
  frame velocity = translation + Omega x X); ABSOLUTE u_r = R_r^T R_d u_d
  (Sec. 2.3.1 eq. "velocity_non", with Q = R^T).  Pressure passes unchanged.
* ``mlp_*`` -- forward/backward of the 3-64-64-3 SiLU guess network in FP64.
* ``face_fluxes``, ``mass_correct`` -- contravariant fluxes U = u . S through receiver faces (Sec. 2.1
  eq. "flux") and the mass-conservation correction over closed interfaces (Sec. 2.4 "Mass conservation").

Parity pins live in ``tests/test_oracle_pins.py``.  The config-level donor
results have no printed values in the paper: "parity unpinned" beyond the
invariants those tests check (closed forms, linear exactness, partition of
unity, affine-cell face distances, rigid-frame identities, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ovs_oracle.c")
_LIB = os.path.join(_HERE, "libovs_oracle.so")

STATUS_FOUND = 0
STATUS_ORPHAN = 1
STATUS_BADINPUT = 2


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (plain gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _OGrid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("per", ctypes.c_int32 * 3),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("iblank", ctypes.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        L.og_num_cells.restype = ctypes.c_int64
        L.og_num_cells.argtypes = [P]
        L.og_num_threads.restype = ctypes.c_int
        L.og_set_num_threads.argtypes = [ctypes.c_int]
        L.og_set_num_threads.restype = None
        L.og_bins_build.restype = P
        L.og_bins_build.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.og_bins_free.argtypes = [P]
        L.og_bins_nreg.restype = ctypes.c_int64
        L.og_bins_nreg.argtypes = [P]
        L.og_search.argtypes = [P, P, ctypes.c_int, ctypes.c_int64, P, P, P, P, P]
        L.og_newton_hex.restype = ctypes.c_int
        L.og_newton_hex.argtypes = [P, P, P, P]
        L.og_surface_inside.argtypes = [ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64, P, P]
        L.og_cell_nodes.argtypes = [P, ctypes.c_int64, P]
        L.og_shape.argtypes = [P, P]
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    return lib().og_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's later parallel loops (n <= 0: one per processor); for timing only."""
    lib().og_set_num_threads(int(n))


class OracleGrid:
    """A donor grid as the oracle sees it (FP64 node coordinates in the grid's own frame)."""

    def __init__(self, dims: Sequence[int], periodic: Sequence[bool], x, y, z, bins: Optional[Sequence[int]] = None):
        self.dims = tuple(int(d) for d in dims)
        self.periodic = tuple(bool(p) for p in periodic)
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        self.z = np.ascontiguousarray(z, dtype=np.float64)
        self._s = _OGrid()
        for d in range(3):
            self._s.n[d] = self.dims[d]
            self._s.per[d] = int(self.periodic[d])
        self._s.x, self._s.y, self._s.z = _ptr(self.x), _ptr(self.y), _ptr(self.z)
        self.cell_dims = tuple(n if p else n - 1 for n, p in zip(self.dims, self.periodic))
        self.n_cells = int(np.prod(self.cell_dims))
        if bins is None:
            bins = tuple(max(1, c // 2) for c in self.cell_dims)
        self._bins = lib().og_bins_build(ctypes.byref(self._s), *[int(b) for b in bins])

    @classmethod
    def from_gen(cls, g, bins=None) -> "OracleGrid":
        return cls(g.dims, g.periodic, g.x, g.y, g.z, bins=bins)

    def set_iblank(self, iblank=None):
        """Per-node mask (0 = blanked: a hole point, never a donor node), or None for every node active.  A cell
        with a blanked corner is never a donor (Sec. 2.4); the search moves on to the next cell, then the next
        grid of the priority list."""
        if iblank is None:
            self.iblank = None
            self._s.iblank = None
        else:
            self.iblank = np.ascontiguousarray(np.asarray(iblank) != 0, dtype=np.uint8)
            assert self.iblank.size == int(np.prod(self.dims))
            self._s.iblank = self.iblank.ctypes.data

    def __del__(self):
        if getattr(self, "_bins", None) and _lib is not None:
            _lib.og_bins_free(self._bins)
            self._bins = None

    @property
    def n_registrations(self) -> int:
        return lib().og_bins_nreg(self._bins)

    def cell_nodes(self, cell: int) -> np.ndarray:
        out = np.zeros(8, dtype=np.int64)
        lib().og_cell_nodes(ctypes.byref(self._s), int(cell), _ptr(out))
        return out

    def search(self, pts: np.ndarray, brute: bool = False):
        """Donor search of donor-frame points (n,3).  Returns (cell int64 [-1 none, -2 non-finite],
        xi (n,3), corner node ids (n,8), weights (n,8))."""
        p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
        n = p.shape[0]
        cell = np.empty(n, dtype=np.int64)
        xi = np.empty((n, 3), dtype=np.float64)
        nodes = np.empty((n, 8), dtype=np.int64)
        w = np.empty((n, 8), dtype=np.float64)
        if n:
            lib().og_search(ctypes.byref(self._s), self._bins, int(bool(brute)), n, _ptr(p), _ptr(cell), _ptr(xi),
                            _ptr(nodes), _ptr(w))
        return cell, xi, nodes, w


def newton_hex(X: np.ndarray, p: np.ndarray):
    """FP64 Newton inversion on one hexahedron X (8,3) (corner a = di+2dj+4dk).  Returns (converged, xi, iters)."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(8, 3)
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(3)
    xi = np.zeros(3)
    it = ctypes.c_int(0)
    ok = lib().og_newton_hex(_ptr(X), _ptr(p), _ptr(xi), ctypes.byref(it))
    return bool(ok), xi, it.value


def surface_inside(V: np.ndarray, T: np.ndarray, P: np.ndarray) -> np.ndarray:
    """Hole cutting (Sec. 2.2.1): 1 where a point (n, 3) is inside the closed triangulated surface (vertices
    V (nv, 3), triangles T (nt, 3) of vertex ids), by the parity of the crossings of a ray along the
    surface's shortest bounding-box axis (the first such axis on a tie), every triangle tested; the tie
    rules are in ovs_oracle.c (og_surface_inside)."""
    V = np.ascontiguousarray(V, dtype=np.float64).reshape(-1, 3)
    T = np.ascontiguousarray(T, dtype=np.int32).reshape(-1, 3)
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(len(P), dtype=np.uint8)
    lib().og_surface_inside(len(V), _ptr(V), len(T), _ptr(T), len(P), _ptr(P), _ptr(out))
    return out


def shape(xi: np.ndarray) -> np.ndarray:
    """Trilinear weights N_a(xi), a = di + 2dj + 4dk (Sec. 2.2.6, (a-1) read as (1-a))."""
    xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(3)
    N = np.zeros(8)
    lib().og_shape(_ptr(xi), _ptr(N))
    return N


# ----------------------------------------------------------------------------- frames
@dataclass
class Frame:
    R: np.ndarray  # body -> inertial
    c: np.ndarray
    V: np.ndarray
    omega: np.ndarray


def frame_of(m) -> Frame:
    return Frame(np.asarray(m.R, float), np.asarray(m.c, float), np.asarray(m.V, float), np.asarray(m.omega, float))


def to_inertial(f: Frame, x: np.ndarray) -> np.ndarray:
    """x_in = R x + c (Sec. 2.1, Fig. "non-inertial"), evaluated in a fixed order, each product and sum rounded
    once: x_in_i = ((R_i0 x_0 + R_i1 x_1) + R_i2 x_2) + c_i.  The order defines the FP64 point every donor and
    hole-cut decision is taken on (the reading of "the point in the donor frame" down to the last bit)."""
    x = np.asarray(x, dtype=np.float64)
    shape, x = x.shape, x.reshape(-1, 3)
    R, c = f.R, f.c
    with np.errstate(invalid="ignore", over="ignore"):
        cols = [((R[i, 0] * x[:, 0] + R[i, 1] * x[:, 1]) + R[i, 2] * x[:, 2]) + c[i] for i in range(3)]
    return np.stack(cols, axis=1).reshape(shape)


def to_frame(f: Frame, x_in: np.ndarray) -> np.ndarray:
    """x_body = R^T (x_in - c), in the fixed order x_body_i = (R_0i d_0 + R_1i d_1) + R_2i d_2, d = x_in - c."""
    x_in = np.asarray(x_in, dtype=np.float64)
    shape, x_in = x_in.shape, x_in.reshape(-1, 3)
    R, c = f.R, f.c
    with np.errstate(invalid="ignore", over="ignore"):
        d = [x_in[:, k] - c[k] for k in range(3)]
        cols = [(R[0, i] * d[0] + R[1, i] * d[1]) + R[2, i] * d[2] for i in range(3)]
    return np.stack(cols, axis=1).reshape(shape)


def frame_map(f_r: Frame, f_d: Frame, x_r: np.ndarray):
    """Receiver-frame points -> (inertial, donor-frame)."""
    x_in = to_inertial(f_r, x_r)
    return x_in, to_frame(f_d, x_in)


# ----------------------------------------------------------------------------- assemble / interpolate
@dataclass
class Donors:
    grid: np.ndarray  # int32 donor grid index, -1 none
    cell: np.ndarray  # int64 donor cell id, -1 none
    xi: np.ndarray  # (n,3) float64, NaN when none
    status: np.ndarray  # uint8
    nodes: np.ndarray  # (n,8) corner node ids
    w: np.ndarray  # (n,8) weights
    x_in: np.ndarray  # (n,3) inertial positions of the query points


def assemble(grids: List[OracleGrid], frames: List[Frame], receiver_xyz: np.ndarray, receiver: int,
             node_ids: np.ndarray, donors: Sequence[int], brute: bool = False) -> Donors:
    """Donors of the receiver nodes ``node_ids`` from the grids ``donors`` in priority order.

    receiver_xyz: (n_nodes,3) receiver-grid node coordinates in the receiver's frame."""
    ids = np.asarray(node_ids, dtype=np.int64)
    n = ids.shape[0]
    x_r = receiver_xyz[ids]
    f_r = frames[receiver]
    x_in = to_inertial(f_r, x_r)
    out = Donors(np.full(n, -1, np.int32), np.full(n, -1, np.int64), np.full((n, 3), np.nan),
                 np.full(n, STATUS_ORPHAN, np.uint8), np.full((n, 8), -1, np.int64), np.zeros((n, 8)), x_in)
    bad = ~np.all(np.isfinite(x_in), axis=1)
    out.status[bad] = STATUS_BADINPUT
    todo = np.nonzero(~bad)[0]
    for gd in donors:
        if todo.size == 0:
            break
        x_d = to_frame(frames[gd], x_in[todo])
        cell, xi, nodes, w = grids[gd].search(x_d, brute=brute)
        hit = cell >= 0
        q = todo[hit]
        out.grid[q] = gd
        out.cell[q] = cell[hit]
        out.xi[q] = xi[hit]
        out.nodes[q] = nodes[hit]
        out.w[q] = w[hit]
        out.status[q] = STATUS_FOUND
        todo = todo[~hit]
    return out


def interpolate(d: Donors, fields: List[dict], frames: List[Frame], receiver: int, mode: str = "relative"):
    """Interpolated (u, v, w, p) at the query points, in the receiver's frame (FP64).  Points without a donor
    get 0."""
    n = d.grid.shape[0]
    out = np.zeros((4, n))
    f_r = frames[receiver]
    for gd in np.unique(d.grid[d.grid >= 0]):
        q = np.nonzero(d.grid == gd)[0]
        f = fields[gd]
        vals = []
        for name in ("u", "v", "w", "p"):
            arr = np.asarray(f[name], dtype=np.float64)
            vals.append(np.sum(d.w[q] * arr[d.nodes[q]], axis=1))
        u_d = np.stack(vals[:3], axis=1)
        f_d = frames[gd]
        if mode == "relative":
            x_in = d.x_in[q]
            u_in = u_d @ f_d.R.T + f_d.V + np.cross(f_d.omega, x_in - f_d.c)
            u_r = (u_in - f_r.V - np.cross(f_r.omega, x_in - f_r.c)) @ f_r.R
        elif mode == "absolute":
            u_r = (u_d @ f_d.R.T) @ f_r.R
        else:
            raise ValueError(mode)
        out[0, q], out[1, q], out[2, q] = u_r[:, 0], u_r[:, 1], u_r[:, 2]
        out[3, q] = vals[3]
    return out


# ----------------------------------------------------------------------------- guess network (FP64)
def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def mlp_forward(params: dict, x: np.ndarray):
    """3 -> H -> H -> 3 network: h1 = silu(x W1^T + b1), h2 = silu(h1 W2^T + b2), y = h2 W3^T + b3.
    W1 (H,3), W2 (H,H), W3 (3,H).  Returns y and the cache for the backward pass."""
    z1 = x @ params["W1"].T + params["b1"]
    h1 = silu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = silu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    return y, (x, z1, h1, z2, h2)


def mlp_loss_grads(params: dict, x: np.ndarray, target: np.ndarray):
    """Mean squared error L = mean over samples and outputs of (y - t)^2 and its gradients (chain rule)."""
    y, (x, z1, h1, z2, h2) = mlp_forward(params, x)
    n = x.shape[0]
    r = y - target
    L = float(np.mean(r * r))
    gy = 2.0 * r / (n * 3)
    g = {}
    g["W3"] = gy.T @ h2
    g["b3"] = gy.sum(axis=0)
    gh2 = gy @ params["W3"]
    gz2 = gh2 * dsilu(z2)
    g["W2"] = gz2.T @ h1
    g["b2"] = gz2.sum(axis=0)
    gh1 = gz2 @ params["W2"]
    gz1 = gh1 * dsilu(z1)
    g["W1"] = gz1.T @ x
    g["b1"] = gz1.sum(axis=0)
    return L, g


def adam_step(params: dict, grads: dict, m: dict, v: dict, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of every parameter, in place; t counts from 1."""
    for k in params:
        m[k] = b1 * m[k] + (1 - b1) * grads[k]
        v[k] = b2 * v[k] + (1 - b2) * grads[k] ** 2
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)


# ----------------------------------------------------------------------------- fluxes at the receivers
# Sec. 2.1 eq. "flux": the contravariant flux U^r = u_q xi^r_q / J through a face of constant xi^r, where
# xi^r_q / J is that face's area vector (per unit of the other two curvilinear coordinates).  On a structured grid
# a face is a quadrilateral of four nodes; its area vector is half the cross product of its diagonals (the
# vector area of the bilinear face), and the velocity on it is the mean of its four corners (Sec. 2.3.1, last
# sentence: the flux of each recipient face from the interpolated velocities).
# Sec. 2.4 "Mass conservation": the fluxes through a closed interface must sum to zero; the imbalance of the
# reconstructed fluxes is removed by a correction.  Reading (the paper defers the details to its earlier work):
# the net outward flux is subtracted from the faces in proportion to their areas.
def face_nodes(dims, periodic, face_id: int):
    """Face id = 3 * (node id of its base corner) + d: the face of constant index along axis d spanned by the
    two axes a = d+1, b = d+2 (mod 3).  Its corners in order: base, base + e_a, base + e_a + e_b, base + e_b (node
    ids, wrapped on periodic axes).  Returns None if the face leaves the grid."""
    n = list(dims)
    node, d = divmod(int(face_id), 3)
    ijk = [node % n[0], (node // n[0]) % n[1], node // (n[0] * n[1])]
    a, b = (d + 1) % 3, (d + 2) % 3
    out = []
    for da, db in ((0, 0), (1, 0), (1, 1), (0, 1)):
        q = list(ijk)
        q[a] += da
        q[b] += db
        for m in range(3):
            if q[m] == n[m]:
                if not periodic[m]:
                    return None
                q[m] = 0
        out.append(q[0] + n[0] * (q[1] + n[1] * q[2]))
    return out


def face_area_vector(xyz: np.ndarray, corners) -> np.ndarray:
    """Half the cross product of the diagonals (corner 2 - corner 0) x (corner 3 - corner 1)."""
    x0, x1, x2, x3 = (xyz[c] for c in corners)
    return 0.5 * np.cross(x2 - x0, x3 - x1)


def face_fluxes(dims, periodic, xyz: np.ndarray, vel: np.ndarray, faces) -> np.ndarray:
    """U_f = (mean of the corner velocities) . S_f for each face id (vel: (n_nodes, 3) in the grid's frame)."""
    out = np.zeros(len(faces))
    for k, f in enumerate(faces):
        c = face_nodes(dims, periodic, f)
        out[k] = np.dot(vel[c].mean(axis=0), face_area_vector(xyz, c))
    return out


def mass_correct(dims, periodic, xyz: np.ndarray, flux: np.ndarray, faces, signs, surf_start):
    """For each closed surface s (faces surf_start[s] .. surf_start[s+1]-1, sign +1 where the face's area vector
    points out of the enclosed region): net = sum of sign * U, A = sum of |S|; each face's flux becomes
    U - sign * net * |S| / A, so that the corrected net flux is zero.  Returns (corrected fluxes, nets, areas)."""
    flux = np.array(flux, dtype=np.float64)
    nets, areas = [], []
    for s in range(len(surf_start) - 1):
        sl = slice(surf_start[s], surf_start[s + 1])
        mag = np.array([np.linalg.norm(face_area_vector(xyz, face_nodes(dims, periodic, f))) for f in faces[sl]])
        sg = np.asarray(signs[sl], dtype=np.float64)
        net = float(np.sum(sg * flux[sl]))
        A = float(np.sum(mag))
        flux[sl] = flux[sl] - sg * net * mag / A
        nets.append(net)
        areas.append(A)
    return flux, np.array(nets), np.array(areas)
