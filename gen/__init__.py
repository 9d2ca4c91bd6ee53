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
    U = np.meshgrid(*u, indexing="ij")
    S = np.meshgrid(*s, indexing="ij")
    bump = np.sin(2 * np.pi * S[0]) * np.sin(2 * np.pi * S[1]) * np.sin(2 * np.pi * S[2])
    coords = []
    for d in range(3):
        L = hi[d] - lo[d]
        h = L / (n[d] - 1)
        coords.append(flat(lo[d] + L * U[d] + pert_h * h * bump))
    return Grid(name, tuple(n), (False, False, False), *coords, role=0)


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


# ----------------------------------------------------------------------------
# fringe-set construction (input selection)
# ----------------------------------------------------------------------------
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


CONFIGS = {0: config0, 1: config1, 2: config2}


def config(i: int) -> Scenario:
    return CONFIGS[i]()
