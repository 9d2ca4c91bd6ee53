"""Seeded synthetic inputs for the overset assembly + interpolation path.

This module builds INPUTS only: curvilinear grids (node coordinates in each
grid's own frame), rigid motions (R, c, V, omega per grid and time step),
fringe (query) point sets, and node fields u, v, w, p.  It contains none of
the method's arithmetic (no donor search, no Newton inversion, no weights, no
interpolation, no velocity transform): the oracle (``oracle/``) and the CUDA
library both consume what is built here and share nothing else.

Workload shapes follow the paper's set-ups: a background grid in the inertial
frame and body-fitted overset grids that move rigidly with their bodies
(Sec. 2.1, Fig. "non-inertial"), fringe points on the outer boundary layers of
each overset grid and background nodes inside an overset grid's hull
(Sec. 2.2.3 item 1), and the school-of-fish geometry of Sec. 3.5
(carangiform midline with quadratic amplitude envelope, diamond offsets).

Conventions
-----------
* Node arrays are flattened with i fastest: ``node = i + ni*(j + nj*k)``.
* ``R`` maps body-frame components to inertial components; ``c`` is the body
  origin in the inertial frame; ``V`` and ``omega`` are the frame's
  translational and angular velocity in inertial components.
* Seeds: numpy PCG64 with seed ``1910093150 + config_index``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np

SEED_BASE = 1910093150


# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------
@dataclass
class Grid:
    """One structured curvilinear grid, coordinates in its own frame."""

    name: str
    dims: tuple  # (ni, nj, nk) node counts
    periodic: tuple  # (bool, bool, bool): axis wraps (last node connects to first)
    x: np.ndarray  # float64, (ni*nj*nk,), i fastest
    y: np.ndarray
    z: np.ndarray
    role: int = 1  # 0 background (inertial), 1 body (moving frame)
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        ni, nj, nk = self.dims
        return ni * nj * nk

    @property
    def cell_dims(self) -> tuple:
        return tuple(n if p else n - 1 for n, p in zip(self.dims, self.periodic))

    @property
    def n_cells(self) -> int:
        ci, cj, ck = self.cell_dims
        return ci * cj * ck

    def xyz(self) -> np.ndarray:
        return np.stack([self.x, self.y, self.z], axis=1)


@dataclass
class Motion:
    R: np.ndarray  # (3,3) body -> inertial
    c: np.ndarray  # (3,)  body origin, inertial
    V: np.ndarray  # (3,)  translational velocity, inertial
    omega: np.ndarray  # (3,) angular velocity, inertial

    @staticmethod
    def identity() -> "Motion":
        return Motion(np.eye(3), np.zeros(3), np.zeros(3), np.zeros(3))


@dataclass
class FringeSet:
    receiver: int  # receiver grid index
    node_ids: np.ndarray  # int32 receiver node ids
    donors: List[int]  # donor grid indices in priority order
    kind: str = ""  # label: "body->bg", "bg->body", "body->body", ...


@dataclass
class Scenario:
    name: str
    grids: List[Grid]
    fields: List[dict]  # per grid: {"u","v","w","p"} arrays (field_dtype)
    field_dtype: type
    dt: float
    nsteps: int
    motion_fn: Callable[[int], List[Motion]]
    sets_fn: Callable[[int, List[Motion]], List[FringeSet]]
    meta: dict = field(default_factory=dict)

    def motion(self, step: int) -> List[Motion]:
        return self.motion_fn(step)

    def fringe_sets(self, step: int, motions: Optional[List[Motion]] = None) -> List[FringeSet]:
        if motions is None:
            motions = self.motion(step)
        return self.sets_fn(step, motions)


# ----------------------------------------------------------------------------
# small helpers (input construction only)
# ----------------------------------------------------------------------------
def rng_for(config_index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + config_index))


def flat(a: np.ndarray) -> np.ndarray:
    """(ni,nj,nk) array -> flat array with i fastest."""
    return np.ascontiguousarray(a.ravel(order="F"))


def euler_zyx(alpha: float, beta: float, gamma: float) -> np.ndarray:
    """Intrinsic z-y-x Euler rotation R = Rz(alpha) Ry(beta) Rx(gamma)."""
    ca, sa = np.cos(alpha), np.sin(alpha)
    cb, sb = np.cos(beta), np.sin(beta)
    cg, sg = np.cos(gamma), np.sin(gamma)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1.0]])
    Ry = np.array([[cb, 0, sb], [0, 1.0, 0], [-sb, 0, cb]])
    Rx = np.array([[1.0, 0, 0], [0, cg, -sg], [0, sg, cg]])
    return Rz @ Ry @ Rx


def axis_angle(axis: np.ndarray, angle: float) -> np.ndarray:
    """Rotation by ``angle`` about unit ``axis`` (Rodrigues)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def random_unit(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def tanh_cluster_centre(n: int, beta: float) -> np.ndarray:
    """Node positions on [0,1] clustered toward 1/2: x(s) = 1/2 + artanh((2s-1) tanh b)/(2b)."""
    s = np.arange(n) / (n - 1)
    return 0.5 + np.arctanh((2 * s - 1) * np.tanh(beta)) / (2 * beta)


def tanh_cluster_wall(n: int, beta: float) -> np.ndarray:
    """Node positions on [0,1] clustered toward 0: t(s) = 1 + tanh(b (s-1)) / tanh(b)."""
    s = np.arange(n) / (n - 1)
    return 1.0 + np.tanh(beta * (s - 1.0)) / np.tanh(beta)


def smooth_field(rng: np.random.Generator, pts: np.ndarray) -> np.ndarray:
    """q(x) = c0 + c.x + sum_{m=1..3} b_m sin(2 pi k_m.x + phi_m), seeded coefficients."""
    c0 = rng.uniform(-1, 1)
    c = rng.uniform(-1, 1, size=3)
    q = c0 + pts @ c
    for _ in range(3):
        b = rng.uniform(0, 0.1)
        k = rng.integers(1, 4, size=3).astype(np.float64)
        phi = rng.uniform(0, 2 * np.pi)
        q = q + b * np.sin(2 * np.pi * (pts @ k) + phi)
    return q


def make_fields(rng: np.random.Generator, grids: Sequence[Grid], dtype) -> List[dict]:
    out = []
    for g in grids:
        pts = g.xyz()
        out.append({name: smooth_field(rng, pts).astype(dtype) for name in ("u", "v", "w", "p")})
    return out


# ----------------------------------------------------------------------------
# grid builders
# ----------------------------------------------------------------------------
def cartesian_grid(name: str, n: Sequence[int], lo: Sequence[float], hi: Sequence[float], role: int = 0) -> Grid:
    axes = [lo[d] + (hi[d] - lo[d]) * np.arange(n[d]) / (n[d] - 1) for d in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    return Grid(name, tuple(n), (False, False, False), flat(X), flat(Y), flat(Z), role)


def perturbed_box_grid(n: int, side: float, amp_h: float) -> Grid:
    """Body box of ``side`` centred at the body origin, n^3 nodes, each node displaced
    (equally in x, y, z) by amp_h*h*sin(2 pi X) sin(2 pi Y) sin(2 pi Z), with (X,Y,Z) the node's
    unperturbed position shifted by +1/2 (its position before the rigid rotation)."""
    h = side / (n - 1)
    a = -side / 2 + side * np.arange(n) / (n - 1)
    X, Y, Z = np.meshgrid(a, a, a, indexing="ij")
    d = amp_h * h * np.sin(2 * np.pi * (X + 0.5)) * np.sin(2 * np.pi * (Y + 0.5)) * np.sin(2 * np.pi * (Z + 0.5))
    return Grid("box32", (n, n, n), (False, False, False), flat(X + d), flat(Y + d), flat(Z + d), 1)


def stretched_background(n: Sequence[int], lo: Sequence[float], hi: Sequence[float], beta: float,
                         cluster_axis: int, pert_h: float, name: str = "bg") -> Grid:
    """Background on the box [lo,hi]: uniform on two axes, tanh-clustered toward the centre plane
    on ``cluster_axis``, plus pert_h*h*prod_k sin(2 pi s_k) added to every coordinate
    (s_k = index/(n_k-1), h = 1/(n_min-1) scaled by the box size; it vanishes on the boundary)."""
    s = [np.arange(n[d]) / (n[d] - 1) for d in range(3)]
    u = [tanh_cluster_centre(n[d], beta) if d == cluster_axis else s[d] for d in range(3)]
    # arrays shaped (nk, nj, ni) in C order, so that ravel() is the i-fastest node order
    shape = [(1, 1, n[0]), (1, n[1], 1), (n[2], 1, 1)]
    sb = [np.sin(2 * np.pi * s[d]).reshape(shape[d]) for d in range(3)]
    bump = (sb[0] * sb[1]) * sb[2]
    coords = []
    axes, pert = [], []
    for d in range(3):
        L = hi[d] - lo[d]
        h = L / (n[d] - 1)
        c = lo[d] + L * u[d].reshape(shape[d])
        coords.append(np.ascontiguousarray((c + pert_h * h * bump).ravel()))
        axes.append(lo[d] + L * u[d])
        pert.append(abs(pert_h) * h)
    return Grid(name, tuple(n), (False, False, False), *coords, role=0, meta=dict(axes=axes, pert=pert))


def box_candidates(bg: Grid, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Node ids of a stretched background whose position lies in the axis-aligned box [lo, hi]: index ranges
    from the unperturbed axes (every node lies within ``pert`` of its axis value), then the exact test."""
    rng = []
    for d in range(3):
        ax = bg.meta["axes"][d]
        a = int(np.searchsorted(ax, lo[d] - bg.meta["pert"][d], side="left"))
        b = int(np.searchsorted(ax, hi[d] + bg.meta["pert"][d], side="right"))
        rng.append(np.arange(a, b, dtype=np.int64))
    ni, nj, _ = bg.dims
    ids = (rng[0][:, None, None] + ni * (rng[1][None, :, None] + nj * rng[2][None, None, :])).ravel()
    if ids.size == 0:
        return ids
    m = ((bg.x[ids] >= lo[0]) & (bg.x[ids] <= hi[0]) & (bg.y[ids] >= lo[1]) & (bg.y[ids] <= hi[1]) &
         (bg.z[ids] >= lo[2]) & (bg.z[ids] <= hi[2]))
    return np.sort(ids[m])


def ellipsoid_ogrid(na: int, npol: int, nr: int, semi: Sequence[float], r_out: float, beta_r: float) -> Grid:
    """Body-fitted O-grid around an ellipsoid with semi-axes ``semi`` (polar axis = body x).

    i: azimuth phi_i = 2 pi i/na (periodic); j: polar theta_j = pi (j+1/2)/npol (the two polar caps
    of half-angle pi/(2 npol) are not covered); k: radial, tanh-clustered toward the surface, from the
    ellipsoid to the sphere of radius r_out."""
    phi = 2 * np.pi * np.arange(na) / na
    th = np.pi * (np.arange(npol) + 0.5) / npol
    t = tanh_cluster_wall(nr, beta_r)
    P, T, Tk = np.meshgrid(phi, th, t, indexing="ij")
    dx = np.cos(T)
    dy = np.sin(T) * np.cos(P)
    dz = np.sin(T) * np.sin(P)
    re = 1.0 / np.sqrt((dx / semi[0]) ** 2 + (dy / semi[1]) ** 2 + (dz / semi[2]) ** 2)
    r = re + (r_out - re) * Tk
    meta = dict(kind="ogrid", semi=tuple(semi), r_out=r_out, t=t, npol=npol)
    return Grid("ogrid", (na, npol, nr), (True, False, False), flat(r * dx), flat(r * dy), flat(r * dz), 1, meta)


def body_surface(g: Grid):
    """The closed triangulated surface of an O-grid's body (its wall layer k = 0 closed by fans to the two pole
    points), in the grid's own frame: vertices (nv, 3) float64 and triangles (nt, 3) int32 vertex ids."""
    na, npol, _ = g.dims
    ring = np.stack([g.x, g.y, g.z], axis=1)[: na * npol]  # k = 0 layer, node i + na j
    kind = g.meta.get("kind")
    if kind == "ogrid":
        a = g.meta["semi"][0]
        poles = np.array([[a, 0.0, 0.0], [-a, 0.0, 0.0]])  # j = 0 lies at +x, j = npol - 1 at -x
    elif kind == "fish":
        ph = g.meta["phase"]
        poles = np.array([[-0.5, float(fish_midline(np.array([0.0]), ph)[0]), 0.0],
                          [0.5, float(fish_midline(np.array([1.0]), ph)[0]), 0.0]])
    else:
        raise ValueError("body_surface: not an O-grid")
    V = np.concatenate([ring, poles])
    i = np.arange(na)
    ip = (i + 1) % na
    tris = []
    for j in range(npol - 1):
        a0, a1, b0, b1 = i + na * j, ip + na * j, i + na * (j + 1), ip + na * (j + 1)
        tris.append(np.stack([a0, a1, b1], axis=1))
        tris.append(np.stack([a0, b1, b0], axis=1))
    A, B = na * npol, na * npol + 1
    tris.append(np.stack([np.full(na, A), ip, i], axis=1))
    tris.append(np.stack([np.full(na, B), i + na * (npol - 1), ip + na * (npol - 1)], axis=1))
    return V, np.concatenate(tris).astype(np.int32)


# ----------------------------------------------------------------------------
# fringe-set construction (input selection)
# ----------------------------------------------------------------------------
def index_box_surface(dims: Sequence[int], periodic: Sequence[bool], lo: Sequence[int], hi: Sequence[int]):
    """The closed surface of the index box of nodes lo[m] .. hi[m] (cells lo[m] .. hi[m]-1) as faces (id = 3 * base
    node + d: the face of constant index along d spanned by the axes d+1, d+2 mod 3) with signs +1 on the box's
    upper-index faces and -1 on its lower ones (outward on a right-handed grid).  An axis given as lo = 0,
    hi = n on a periodic axis wraps around: it has no end faces.  Returns (faces int64, signs int8)."""
    n = list(dims)
    faces, signs = [], []
    for d in range(3):
        a, b = (d + 1) % 3, (d + 2) % 3
        if periodic[d] and lo[d] == 0 and hi[d] == n[d]:
            continue
        for side, sgn in ((lo[d], -1), (hi[d], 1)):
            for ib in range(lo[b], hi[b]):
                for ia in range(lo[a], hi[a]):
                    q = [0, 0, 0]
                    q[d], q[a], q[b] = side, ia, ib
                    faces.append(3 * (q[0] + n[0] * (q[1] + n[1] * q[2])) + d)
                    signs.append(sgn)
    return np.array(faces, dtype=np.int64), np.array(signs, dtype=np.int8)


def outer_layers(g: Grid, layers: int, axes: Sequence[int]) -> np.ndarray:
    """Node ids within ``layers`` nodes of the low/high boundary on any of ``axes``
    (periodic axes have no boundary and are skipped)."""
    ni, nj, nk = g.dims
    idx = np.meshgrid(np.arange(ni), np.arange(nj), np.arange(nk), indexing="ij")
    mask = np.zeros(g.dims, dtype=bool)
    for d in axes:
        if g.periodic[d]:
            continue
        n = g.dims[d]
        mask |= (idx[d] < layers) | (idx[d] >= n - layers)
    ids = np.arange(ni * nj * nk, dtype=np.int64).reshape(g.dims, order="F")
    return flat(ids)[flat(mask)].astype(np.int32)


def radial_layers(g: Grid, layers: int) -> np.ndarray:
    """Node ids on the outermost ``layers`` k-layers."""
    ni, nj, nk = g.dims
    ids = np.arange(ni * nj * nk, dtype=np.int64).reshape((ni, nj, nk), order="F")
    return np.ascontiguousarray(ids[:, :, nk - layers:].ravel(order="F")).astype(np.int32)


def to_body(m: Motion, pts: np.ndarray) -> np.ndarray:
    """Body-frame position of inertial points (used only to select query points)."""
    return (pts - m.c) @ m.R


def inside_box_hull(m: Motion, pts: np.ndarray, half: float) -> np.ndarray:
    p = to_body(m, pts)
    return np.all(np.abs(p) < half, axis=1)


def inside_ogrid_hull(m: Motion, pts: np.ndarray, g: Grid) -> np.ndarray:
    """Inside the O-grid's outer sphere shrunk to node layer nk-3 and outside the ellipsoid."""
    meta = g.meta
    p = to_body(m, pts)
    r = np.linalg.norm(p, axis=1)
    d = p / np.maximum(r, 1e-300)[:, None]
    semi = meta["semi"]
    re = 1.0 / np.sqrt((d[:, 0] / semi[0]) ** 2 + (d[:, 1] / semi[1]) ** 2 + (d[:, 2] / semi[2]) ** 2)
    t_in = meta["t"][-3]
    r_in = re + (meta["r_out"] - re) * t_in
    return (r < r_in) & (r > re)


def bbox_candidates(bg: Grid, centre: np.ndarray, radius: float) -> np.ndarray:
    """Background node ids inside the axis-aligned cube of half-size ``radius`` around ``centre``."""
    lo = centre - radius
    hi = centre + radius
    m = ((bg.x >= lo[0]) & (bg.x <= hi[0]) & (bg.y >= lo[1]) & (bg.y <= hi[1]) & (bg.z >= lo[2]) & (bg.z <= hi[2]))
    return np.nonzero(m)[0].astype(np.int64)


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------
def config0() -> Scenario:
    """Plain method, tiny: uniform Cartesian 64^3 background on [0,1]^3 and a perturbed 32^3 box of side 0.4
    rigidly rotated by seeded z-y-x Euler angles U(0, pi) about its centre (0.5,0.5,0.5).  Fringe: the
    outer 2 node layers of the box (search the background) and the background nodes inside the box
    shrunk by two of its cells (search the box).  FP64 fields.  One step; the frame velocity V, omega is
    seeded so that the velocity transform is exercised."""
    rng = rng_for(0)
    bg = cartesian_grid("bg64", (64, 64, 64), (0, 0, 0), (1, 1, 1), role=0)
    body = perturbed_box_grid(32, 0.4, 0.05)
    R = euler_zyx(*rng.uniform(0, np.pi, size=3))
    c = np.array([0.5, 0.5, 0.5])
    V = rng.uniform(-0.5, 0.5, size=3)
    om = rng.uniform(-2 * np.pi, 2 * np.pi, size=3)
    grids = [bg, body]
    fields = make_fields(rng, grids, np.float64)
    motion_body = Motion(R, c, V, om)
    body_fringe = outer_layers(body, 2, (0, 1, 2))
    hb = 0.4 / 31
    bg_pts = bg.xyz()

    def motion_fn(step: int) -> List[Motion]:
        return [Motion.identity(), motion_body]

    def sets_fn(step: int, motions: List[Motion]) -> List[FringeSet]:
        m = motions[1]
        inside = inside_box_hull(m, bg_pts, 0.2 - 2 * hb)
        bg_ids = np.nonzero(inside)[0].astype(np.int32)
        return [FringeSet(1, body_fringe, [0], "body->bg"), FringeSet(0, bg_ids, [1], "bg->body")]

    return Scenario("cfg0: bg 64^3 Cartesian + rotated perturbed box 32^3", grids, fields, np.float64,
                    dt=0.0, nsteps=1, motion_fn=motion_fn, sets_fn=sets_fn)


def moving_ellipsoid(config_index: int, nbg: int, nsteps: int = 100, dt: float = 1e-3) -> Scenario:
    """Stretched curvilinear background nbg^3 on [0,1]^3 (tanh clustering beta=2 toward y=1/2, 0.1h sinusoidal
    perturbation) and a 96x64x64 O-grid around an ellipsoid (0.2,0.1,0.1) out to r=0.4, rotating at
    2 pi rad/time about a seeded axis and translating at 0.3/time along a seeded direction (centred at
    (0.5,0.5,0.5) at mid-run).  Fringe: O-grid radial layers k in {62,63} (search the background) and the
    background nodes inside the O-grid hull (search the O-grid), recomputed each step.  FP32 fields."""
    rng = rng_for(config_index)
    bg = stretched_background((nbg, nbg, nbg), (0, 0, 0), (1, 1, 1), beta=2.0, cluster_axis=1, pert_h=0.1,
                              name=f"bg{nbg}")
    body = ellipsoid_ogrid(96, 64, 64, (0.2, 0.1, 0.1), 0.4, beta_r=2.0)
    grids = [bg, body]
    fields = make_fields(rng, grids, np.float32)
    axis = random_unit(rng)
    vdir = random_unit(rng)
    R0 = euler_zyx(*rng.uniform(0, np.pi, size=3))
    om = 2 * np.pi * axis
    V = 0.3 * vdir
    T = nsteps * dt
    c0 = np.array([0.5, 0.5, 0.5]) - V * (T / 2)
    body_fringe = radial_layers(body, 2)
    cand = bbox_candidates(bg, np.array([0.5, 0.5, 0.5]), 0.4 + 0.3 * T / 2 + 1e-9)
    cand_pts = bg.xyz()[cand]

    def motion_fn(step: int) -> List[Motion]:
        t = step * dt
        R = axis_angle(axis, 2 * np.pi * t) @ R0
        return [Motion.identity(), Motion(R, c0 + V * t, V.copy(), om.copy())]

    def sets_fn(step: int, motions: List[Motion]) -> List[FringeSet]:
        inside = inside_ogrid_hull(motions[1], cand_pts, body)
        bg_ids = cand[inside].astype(np.int32)
        return [FringeSet(1, body_fringe, [0], "body->bg"), FringeSet(0, bg_ids, [1], "bg->body")]

    return Scenario(f"cfg{config_index}: stretched bg {nbg}^3 + moving ellipsoid O-grid 96x64x64", grids, fields,
                    np.float32, dt=dt, nsteps=nsteps, motion_fn=motion_fn, sets_fn=sets_fn,
                    meta=dict(axis=axis, vdir=vdir))


# ----------------------------------------------------------------------------
# school of fish (Sec. 3.5 geometry, synthetic bodies)
# ----------------------------------------------------------------------------
FISH_WAVELENGTH = 0.95  # lambda / L (Sec. 3.5)
FISH_TAIL_BEAT = 1.0 / (240 * 1.39e-3)  # 240 time steps of dt = 1.39e-3 per tail beat (Sec. 3.5)


def naca0012_half_thickness(s: np.ndarray) -> np.ndarray:
    """Half-thickness of the NACA 4-digit section of 12% thickness at chord fraction s in [0,1] (closed
    trailing edge variant of the last coefficient)."""
    s = np.clip(s, 0.0, 1.0)
    return 0.6 * (0.2969 * np.sqrt(s) - 0.1260 * s - 0.3516 * s ** 2 + 0.2843 * s ** 3 - 0.1036 * s ** 4)


def fish_envelope(s: np.ndarray) -> np.ndarray:
    """Amplitude envelope a(s) = a0 + a1 s + a2 s^2 with (a0, a1, a2) = (0.02, -0.08, 0.16), so that the tail
    (s = 1) reaches the maximum excursion 0.1 L that Sec. 3.5 states."""
    return 0.02 - 0.08 * s + 0.16 * s ** 2


def fish_midline(s: np.ndarray, phase: float) -> np.ndarray:
    """Frozen lateral excursion of the midline, h(s) = a(s) sin(2 pi s / lambda - phase) (Sec. 3.5 at one
    instant)."""
    return fish_envelope(s) * np.sin(2 * np.pi * s / FISH_WAVELENGTH - phase)


# In body lengths.  The hull's axial semi-axis equals the body's (A = 1/2): radial and azimuthal grid edges then
# lie in planes x = const, where the midline shear y += h(x) leaves every corner Jacobian unchanged.
FISH_HULL = dict(A=0.5, B=0.25, C=0.2, height=1.6, beta_r=2.0)


def fish_ogrid(name: str, na: int, npol: int, nr: int, phase: float) -> Grid:
    """Body-fitted O-grid around a fish-like body of length 1 (head at body x = -1/2, tail at +1/2).

    Body: at chord fraction s (head 0, tail 1) the cross-section is an ellipse centred on the midline
    h(s) (lateral, body y) with lateral half-width the NACA0012 half-thickness w(s) and vertical half-height
    1.6 w(s).  Outer boundary: an ellipsoid of semi-axes (A = 1/2, B, C).  The grid of the straight body (h = 0) is
    sheared laterally, y += h(clip(x + 1/2, 0, 1)), at each node's own x: a map of unit Jacobian, so the bent
    grid is as regular as the straight one, and the body surface keeps its cross-sections on the midline.
    i: azimuth th_i = 2 pi i/na (periodic); j: polar angle ph_j = pi (j+1/2)/npol with s = (1 - cos ph)/2 (the
    head and tail caps of half-angle pi/(2 npol) are not covered); k: radial fraction f_k tanh-clustered toward
    the body.  Node = (X, h(X + 1/2) + Bf cos th, Cf sin th) with X = -((1-f)/2 + f A) cos ph, Bf = (1-f) w(s) +
    f B sin ph, Cf = (1-f) 1.6 w(s) + f C sin ph: every k-layer is a surface of ellipses at fixed x, which makes
    the hull test below exact."""
    P = FISH_HULL
    th = 2 * np.pi * np.arange(na) / na
    ph = np.pi * (np.arange(npol) + 0.5) / npol
    f = tanh_cluster_wall(nr, P["beta_r"])
    TH, PH, F = np.meshgrid(th, ph, f, indexing="ij")
    s = 0.5 * (1 - np.cos(PH))
    w = naca0012_half_thickness(s)
    X = -((1 - F) * 0.5 + F * P["A"]) * np.cos(PH)
    Bf = (1 - F) * w + F * P["B"] * np.sin(PH)
    Cf = (1 - F) * P["height"] * w + F * P["C"] * np.sin(PH)
    hx = fish_midline(np.clip(X + 0.5, 0.0, 1.0), phase)
    meta = dict(kind="fish", phase=phase, t=f, npol=npol)
    return Grid(name, (na, npol, nr), (True, False, False), flat(X), flat(hx + Bf * np.cos(TH)),
                flat(Cf * np.sin(TH)), 1, meta)


def inside_fish_layer(p: np.ndarray, phase: float, frac: float) -> np.ndarray:
    """Body-frame points strictly inside the k-layer surface of radial fraction ``frac`` of a fish O-grid
    (frac = 0: the body itself)."""
    P = FISH_HULL
    Af = (1 - frac) * 0.5 + frac * P["A"]
    cph = -p[:, 0] / Af
    ok = np.abs(cph) < 1
    cph = np.clip(cph, -1, 1)
    sph = np.sqrt(1 - cph ** 2)
    s = 0.5 * (1 - cph)
    w = naca0012_half_thickness(s)
    Bf = (1 - frac) * w + frac * P["B"] * sph
    Cf = (1 - frac) * P["height"] * w + frac * P["C"] * sph
    with np.errstate(divide="ignore", invalid="ignore"):
        q = ((p[:, 1] - fish_midline(np.clip(p[:, 0] + 0.5, 0.0, 1.0), phase)) / Bf) ** 2 + (p[:, 2] / Cf) ** 2
    return ok & (Bf > 0) & (Cf > 0) & (q < 1)


def fish_sizes(n: int, lo: Sequence[int], hi: Sequence[int]) -> List[tuple]:
    """n grid sizes linearly spaced from lo to hi (azimuth rounded to a multiple of 8, the others to 4)."""
    out = []
    for q in range(n):
        a = q / max(1, n - 1)
        d = [lo[k] + (hi[k] - lo[k]) * a for k in range(3)]
        out.append((int(round(d[0] / 8) * 8), int(round(d[1] / 4) * 4), int(round(d[2] / 4) * 4)))
    return out


def fish_school(config_index: int, nfish: int, bg_dims: Sequence[int], size_lo: Sequence[int],
                size_hi: Sequence[int], layers: Sequence[float], nsteps: int, dt: float = 1.39e-3) -> Scenario:
    """Diamond school of fish-like O-grids in a stretched curvilinear background (Sec. 3.5 geometry).

    Diamonds of four (front; two sides 0.45 L lateral and 1.45 L posterior; last 2.9 L behind), two side by side
    1.2 L apart (so the hulls of the two inner side fish overlap), one such pair per vertical ``layers`` entry;
    seeded jitter of 0.03 L.  All fish share the
    seeded phase of the frozen midline (no phase difference between swimmers, Sec. 3.5).  Each swims rigidly
    toward -x at a seeded speed U in [0.9, 1.1] with a seeded yaw oscillation of 0.05 rad at the tail-beat
    frequency.  Body grid sizes are spread linearly between ``size_lo`` and ``size_hi`` and assigned in seeded
    order.  Background: box around the school's path, x streamwise, y lateral (tanh clustering beta = 2 toward
    the centre plane, 0.1 h sinusoidal perturbation), z vertical.  Fringe sets per step:
      * each body's outer two radial layers: points inside another body's hull (shrunk to its layer nk-3, outside
        its body) search [those bodies in id order, background], the rest [background];
      * background nodes inside a body's shrunk hull and outside every body, grouped by the bodies containing
        them, search those bodies in id order.
    FP32 fields."""
    rng = rng_for(config_index)
    base = [(0.0, 0.0), (1.45, 0.45), (1.45, -0.45), (2.9, 0.0)]
    pos = []
    for zc in layers:
        for yc in (-0.6, 0.6):
            for (px, py) in base:
                if len(pos) < nfish:
                    pos.append(np.array([px, yc + py, zc]) + rng.uniform(-0.03, 0.03, size=3))
    pos = np.array(pos)
    speed = rng.uniform(0.9, 1.1, size=nfish)
    yaw0 = rng.uniform(-0.05, 0.05, size=nfish)
    yaw_phase = rng.uniform(0, 2 * np.pi, size=nfish)
    phase = float(rng.uniform(0, 2 * np.pi))
    sizes = fish_sizes(nfish, size_lo, size_hi)
    order = rng.permutation(nfish)
    T = nsteps * dt
    P = FISH_HULL
    reach = P["A"] + 0.05
    lo = np.array([pos[:, 0].min() - speed.max() * T - reach - 0.3, pos[:, 1].min() - P["B"] - 0.45,
                   pos[:, 2].min() - P["C"] - 0.3])
    hi = np.array([pos[:, 0].max() + reach + 0.3, pos[:, 1].max() + P["B"] + 0.45, pos[:, 2].max() + P["C"] + 0.3])
    bg = stretched_background(tuple(bg_dims), lo, hi, beta=2.0, cluster_axis=1, pert_h=0.1,
                              name="bg%dx%dx%d" % tuple(bg_dims))
    bodies = [fish_ogrid("fish%d" % q, *sizes[order[q]], phase) for q in range(nfish)]
    grids = [bg] + bodies
    fields = make_fields(rng, grids, np.float32)
    fringes = [radial_layers(b, 2) for b in bodies]
    # inertial half-extents of a hull under yaw |psi| <= 0.1 (|x_b| <= A, |y_b| <= B + max|h| = B + 0.1, |z_b| <= C)
    half = np.array([P["A"] + (P["B"] + 0.1) * 0.1 + 0.01, P["B"] + 0.1 + P["A"] * 0.1 + 0.01, P["C"] + 0.01])
    frac_in = [b.meta["t"][-3] for b in bodies]
    amp = 0.05

    def motion_fn(step: int) -> List[Motion]:
        t = step * dt
        out = [Motion.identity()]
        for q in range(nfish):
            arg = 2 * np.pi * FISH_TAIL_BEAT * t + yaw_phase[q]
            psi = yaw0[q] + amp * np.sin(arg)
            dpsi = amp * 2 * np.pi * FISH_TAIL_BEAT * np.cos(arg)
            R = axis_angle(np.array([0.0, 0.0, 1.0]), psi)
            V = np.array([-speed[q], 0.0, 0.0])
            out.append(Motion(R, pos[q] + V * t, V, np.array([0.0, 0.0, dpsi])))
        return out

    def sets_fn(step: int, motions: List[Motion]) -> List[FringeSet]:
        ms = motions[1:]
        sets: List[FringeSet] = []
        # body fringe: inside other bodies' hulls -> those bodies first, then the background
        for q, b in enumerate(bodies):
            ids = fringes[q]
            pts = (b.xyz()[ids] @ ms[q].R.T) + ms[q].c
            keys = np.zeros(len(ids), dtype=np.int64)
            for r in range(nfish):
                if r == q or np.linalg.norm(ms[r].c - ms[q].c) > 2 * reach:
                    continue
                pb = to_body(ms[r], pts)
                hit = inside_fish_layer(pb, phase, frac_in[r])
                hit[hit] &= ~inside_fish_layer(pb[hit], phase, 0.0)
                keys |= hit.astype(np.int64) << r
            for key in np.unique(keys):
                sel = ids[keys == key]
                don = [1 + r for r in range(nfish) if (int(key) >> r) & 1][:7] + [0]
                sets.append(FringeSet(1 + q, sel.astype(np.int32), don, "body->bg" if key == 0 else "body->body"))
        # background nodes inside hulls, outside every body, grouped by the hulls that hold them
        nodes, bits, solid = [], [], []
        for q in range(nfish):
            cand = box_candidates(bg, ms[q].c - half, ms[q].c + half)
            pb = to_body(ms[q], np.stack([bg.x[cand], bg.y[cand], bg.z[cand]], axis=1))
            hit = inside_fish_layer(pb, phase, frac_in[q])
            body_hit = np.zeros_like(hit)
            body_hit[hit] = inside_fish_layer(pb[hit], phase, 0.0)
            nodes.append(cand[hit])
            bits.append(np.full(int(hit.sum()), 1 << q, dtype=np.int64))
            solid.append(cand[body_hit])
        nodes = np.concatenate(nodes)
        bits = np.concatenate(bits)
        order = np.argsort(nodes, kind="stable")
        nodes, bits = nodes[order], bits[order]
        uniq, start = np.unique(nodes, return_index=True)
        keys = np.bitwise_or.reduceat(bits, start) if len(uniq) else bits
        keep = ~np.isin(uniq, np.concatenate(solid))
        uniq, keys = uniq[keep], keys[keep]
        for key in np.unique(keys):
            sel = uniq[keys == key]
            don = [1 + r for r in range(nfish) if (int(key) >> r) & 1][:8]
            sets.append(FringeSet(0, sel.astype(np.int32), don, "bg->body"))
        return sets

    def iblank_fn(motions: List[Motion]) -> List[np.ndarray]:
        """Hole cut of the step: background nodes inside any fish body are blanked (0); body nodes all active."""
        ms = motions[1:]
        bgmask = np.ones(bg.n_nodes, dtype=np.uint8)
        for q in range(nfish):
            cand = box_candidates(bg, ms[q].c - half, ms[q].c + half)
            pb = to_body(ms[q], np.stack([bg.x[cand], bg.y[cand], bg.z[cand]], axis=1))
            bgmask[cand[inside_fish_layer(pb, phase, 0.0)]] = 0
        return [bgmask] + [np.ones(b.n_nodes, dtype=np.uint8) for b in bodies]

    return Scenario(f"cfg{config_index}: school of {nfish} fish O-grids in a stretched bg "
                    "%dx%dx%d" % tuple(bg_dims), grids, fields, np.float32, dt=dt, nsteps=nsteps,
                    motion_fn=motion_fn, sets_fn=sets_fn,
                    meta=dict(phase=phase, positions=pos, sizes=sizes, iblank_fn=iblank_fn))


def config1() -> Scenario:
    return moving_ellipsoid(1, 128)


def config2() -> Scenario:
    return moving_ellipsoid(2, 256)


def mlp_training_samples(config_index: int, grid: Grid, n_samples: int):
    """Random (cell, xi) draws for training a body grid's guess network: cell uniform over the grid's cells,
    xi uniform on [0,1]^3.  Returns (cells int32, xi float64 (n,3))."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 1000 + config_index))
    cells = rng.integers(0, grid.n_cells, size=n_samples).astype(np.int32)
    xi = rng.random((n_samples, 3))
    return cells, xi


def config3() -> Scenario:
    """8 fish of 48x32x32 .. 128x64x64 in a 384x256x128 background, 200 steps."""
    return fish_school(3, 8, (384, 256, 128), (48, 32, 32), (128, 64, 64), layers=(0.0,), nsteps=200)


def config4() -> Scenario:
    """16 fish of 64^3 .. 160x96x96 (two layers of the 8-fish school 0.6 L apart) in a 512x384x256 background
    (~50M nodes), 1000 steps."""
    return fish_school(4, 16, (512, 384, 256), (64, 64, 64), (160, 96, 96), layers=(-0.3, 0.3), nsteps=1000)


CONFIGS = {0: config0, 1: config1, 2: config2, 3: config3, 4: config4}


def config(i: int) -> Scenario:
    return CONFIGS[i]()
