"""Hole cutting on the GPU (paper Sec. 2.2.1: background nodes inside a moving body's closed surface are blanked)
against the oracle's ray parity:

* every fish surface of the 8-fish school cuts the background nodes near it (all in one launch, the same mask as
  one call per fish); on a seeded sample of the nodes near every fish the GPU's mask equals the oracle's byte for
  byte (both decide on the same FP64 point: the frame maps' fixed order of operations, Sec. 2.1);
* the mask then drives the donor search (blanked donors rejected), which equals the oracle's with that mask.
"""
import numpy as np
import pytest

import gen
import oracle
from harness import GpuScene, OracleScene, compare, split
from paper_1910_09315_gb300 import ovs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def near_body_nodes(bg, m):
    """Background nodes in a box around a fish body (length 1, half-width < 0.2, half-height < 0.12), any yaw."""
    return gen.box_candidates(bg, m.c - np.array([0.56, 0.56, 0.14]), m.c + np.array([0.56, 0.56, 0.14]))


def test_hole_cut_matches_oracle(torch_cuda):
    t = torch_cuda
    sc = gen.config(3)
    m = sc.motion(0)
    scene = GpuScene(sc, max_points=1024)
    scene.set_motion(m)
    bg = sc.grids[0]
    dev = scene.ctx.device
    iblank = t.ones(bg.n_nodes, dtype=t.uint8, device=dev)
    rng = np.random.default_rng(11)
    checked, cut = 0, 0
    surfaces, sids, cands = [], [], []
    for q in range(1, len(sc.grids)):
        V, T = gen.body_surface(sc.grids[q])
        sids.append(scene.ctx.add_surface(scene.ids[q], V, T))
        surfaces.append((q, V, T))
        cands.append(t.as_tensor(near_body_nodes(bg, m[q]).astype(np.int32)).to(dev))
    # all bodies in one launch, and one call per body: the same mask
    scene.ctx.hole_cut_many(sids, scene.ids[0], iblank, cands)
    one_by_one = t.ones_like(iblank)
    for sid, cand in zip(sids, cands):
        scene.ctx.hole_cut(sid, scene.ids[0], one_by_one, nodes=cand)
    scene.ctx.sync()
    mask = iblank.cpu().numpy()
    assert np.array_equal(mask, one_by_one.cpu().numpy())
    # one seeded sample of background nodes, each tested against every surface whose box holds it
    keep = rng.random(bg.n_nodes) < 0.15
    inside_any = np.zeros(bg.n_nodes, dtype=bool)
    sampled = np.zeros(bg.n_nodes, dtype=bool)
    for q, V, T in surfaces:
        cand = near_body_nodes(bg, m[q])
        cand = cand[keep[cand]]
        fb, ft = oracle.frame_of(m[q]), oracle.frame_of(m[0])
        pb = oracle.to_frame(fb, oracle.to_inertial(ft, bg.xyz()[cand]))
        ins = oracle.surface_inside(V, T, pb).astype(bool)
        inside_any[cand[ins]] = True
        sampled[cand] = True
        cut += int(ins.sum())
    s = np.nonzero(sampled)[0]
    got = mask[s] == 0
    want = inside_any[s]
    bad = s[got != want]
    assert bad.size == 0, f"{bad.size} mask bytes differ, first nodes {bad[:8]}"
    checked = len(s)
    assert checked > 100_000 and cut > 5_000


def test_hole_cut_drives_the_donor_search(torch_cuda):
    t = torch_cuda
    sc = gen.config(3)
    m = sc.motion(0)
    fsets = sc.fringe_sets(0, m)
    n = sum(len(s.node_ids) for s in fsets)
    scene = GpuScene(sc, max_points=n + 1024)
    scene.set_motion(m)
    bg = sc.grids[0]
    dev = scene.ctx.device
    iblank = t.ones(bg.n_nodes, dtype=t.uint8, device=dev)
    for q in range(1, len(sc.grids)):
        V, T = gen.body_surface(sc.grids[q])
        sid = scene.ctx.add_surface(scene.ids[q], V, T)
        scene.ctx.hole_cut(sid, scene.ids[0], iblank, nodes=t.as_tensor(near_body_nodes(bg, m[q]).astype(np.int32)).to(dev))
    ovs.ovs_set_iblank(scene.ctx.ctx, scene.ids[0], iblank.data_ptr())
    mask = iblank.cpu().numpy()
    assert (mask == 0).sum() > 10_000
    ref = OracleScene(sc)
    ref.grids[0].set_iblank(mask)
    _, d, out = scene.step(m, fsets)
    res = GpuScene.to_numpy(d, out)
    parts = split(res, [len(s.node_ids) for s in fsets])
    rng = np.random.default_rng(5)
    sample = [np.sort(rng.choice(len(s.node_ids), size=max(1, len(s.node_ids) // 10), replace=False)) for s in fsets]
    oref, frames = ref.step(m, fsets, sample=sample)
    total = 0
    for k, (s, part, (od, oq)) in enumerate(zip(fsets, parts, oref)):
        part = {kk: (v[..., sample[k]] if kk == "q" else v[sample[k]]) for kk, v in part.items()}
        total += compare(part, od, oq, sc, frames, s.receiver, ovs.OVS_F32, label=f"hole-cut set {k}")
    assert total > 50_000


def cube_surface(k):
    """The unit cube's surface, each face split into k x k squares and each square into two triangles along a
    diagonal (vertex coordinates multiples of 1/k: shared edges have identical coordinates)."""
    V, T = [], []
    for a in range(3):
        u, w = (a + 1) % 3, (a + 2) % 3
        for side in (0.0, 1.0):
            base = len(V)
            for j in range(k + 1):
                for i in range(k + 1):
                    p = [0.0, 0.0, 0.0]
                    p[a], p[u], p[w] = side, i / k, j / k
                    V.append(p)
            vid = lambda i, j: base + i + (k + 1) * j
            for j in range(k):
                for i in range(k):
                    T += [(vid(i, j), vid(i + 1, j), vid(i + 1, j + 1)), (vid(i, j), vid(i + 1, j + 1), vid(i, j + 1))]
    return np.array(V), np.array(T, np.int32)


def test_hole_cut_cube_ties_bit_exact(torch_cuda):
    """Points exactly on the cube's faces, edges, vertices and face diagonals (a lattice of spacing 1/16), and
    points at dyadic distances 2^-40 .. 2^-10 off the faces or exactly on them: every coordinate is exact in FP32
    pairs and the motion is the identity, so the GPU's FP64 tie rules see the oracle's points and its mask must
    equal the oracle's everywhere; most of these points sit where the FP32 decisions must defer to FP64."""
    t = torch_cuda
    V, T = cube_surface(4)
    lat = gen.cartesian_grid("lattice", (25, 25, 25), (-0.25, -0.25, -0.25), (1.25, 1.25, 1.25), role=0)
    rng = np.random.default_rng(8)
    m = 4 * 6000
    P = np.empty((m, 3))
    a = rng.integers(0, 3, m)
    side = rng.integers(0, 2, m).astype(np.float64)
    off = np.ldexp(rng.choice([-1.0, 1.0], m), -rng.integers(10, 41, m))
    off[rng.random(m) < 0.1] = 0.0
    for r in range(m):
        q = rng.integers(-(1 << 18), (1 << 20) + (1 << 18), 3) / float(1 << 20)
        q[a[r]] = side[r] + off[r]
        P[r] = q
    near = gen.Grid("near", (m // 4, 2, 2), (False, False, False), P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy(), 0)
    body = gen.cartesian_grid("body", (3, 3, 3), (0.2, 0.2, 0.2), (0.8, 0.8, 0.8), role=1)
    ctx = ovs.Context(max_points=1024)
    ids = [ctx.add_grid(g.x, g.y, g.z, g.dims, g.periodic, g.role) for g in (lat, near, body)]
    for gid in ids:
        ctx.set_motion(gid, np.eye(3), np.zeros(3), np.zeros(3), np.zeros(3))
    sid = ctx.add_surface(ids[2], V, T)
    for g, gid in zip((lat, near), ids):
        iblank = t.ones(g.n_nodes, dtype=t.uint8, device=ctx.device)
        ctx.hole_cut(sid, gid, iblank)
        ctx.sync()
        want = 1 - oracle.surface_inside(V, T, g.xyz())
        got = iblank.cpu().numpy()
        assert np.array_equal(got, want), (g.name, np.nonzero(got != want)[0][:10])
    assert (1 - want).sum() > m // 10 and want.sum() > m // 2
