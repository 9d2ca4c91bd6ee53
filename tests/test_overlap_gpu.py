"""Grids whose cells overlap one another, on the GPU against the oracle.

The fast path takes a donor from the walk alone when no other cell of the grid can hold the point; where cells
overlap, the lowest-id rule needs the exhaustive search of the control cell.  Two cases:
* a folded cell (one node pushed past its neighbours): ovs_create_grid finds it from the corner Jacobians and
  searches that grid exhaustively on its own;
* an annulus whose periodic azimuth wraps around twice: no cell is folded, every point lies in two cells, and only
  the caller knows; with ovs_set_grid_overlap the donors are the oracle's lowest ids.
Donors are compared bit for bit, weights and fields with the tolerances of tests/harness.py.
"""
import numpy as np
import pytest

import gen
from harness import GpuScene, OracleScene, compare, split
from paper_1910_09315_gb300 import ovs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def scenario(donor, receiver, ids, seed):
    grids = [receiver, donor]
    fields = gen.make_fields(np.random.default_rng(seed), grids, np.float64)
    return gen.Scenario("overlap", grids, fields, np.float64, dt=1.0, nsteps=1,
                        motion_fn=lambda s: [gen.Motion.identity(), gen.Motion.identity()],
                        sets_fn=lambda s, m: [gen.FringeSet(0, ids.astype(np.int32), [1], "bg->body")])


def run(sc, overlap=None):
    m = sc.motion(0)
    fsets = sc.fringe_sets(0, m)
    scene = GpuScene(sc, max_points=sum(len(s.node_ids) for s in fsets) + 16, xi_dtype=ovs.OVS_F64)
    if overlap is not None:
        ovs.ovs_set_grid_overlap(scene.ctx.ctx, 1, overlap)
    _, d, out = scene.step(m, fsets)
    res = GpuScene.to_numpy(d, out)
    return scene, fsets, res


def check(sc, fsets, res):
    m = sc.motion(0)
    oref, frames = OracleScene(sc).step(m, fsets)
    parts = split(res, [len(s.node_ids) for s in fsets])
    n = 0
    for k, (s, part, (od, oq)) in enumerate(zip(fsets, parts, oref)):
        n += compare(part, od, oq, sc, frames, s.receiver, ovs.OVS_F64, label=f"overlap set {k}")
    return n


def test_folded_cell_is_found_and_searched_exhaustively(torch_cuda):
    """One node pushed past its neighbour folds the cells around it.  ovs_create_grid counts them and searches
    the grid exhaustively; the donors of points away from the folded cells (where the inverse of a folded cell's
    map, and so the donor rule itself, depends on where Newton starts) are the oracle's."""
    donor = gen.cartesian_grid("d", (9, 9, 9), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), role=1)
    h = 1.0 / 8
    node = 4 + 9 * (4 + 9 * 4)
    donor.x = donor.x.copy()
    donor.x[node] -= 1.6 * h  # past the node before it: the cells around it fold
    recv = gen.cartesian_grid("r", (25, 25, 25), (0.02, 0.02, 0.02), (0.98, 0.98, 0.98), role=0)
    far = np.max(np.abs(recv.xyz() - 0.5), axis=1) > 2.05 * h  # outside the folded cells' box [2h, 6h]^3
    sc = scenario(donor, recv, np.nonzero(far)[0], 5)
    scene, fsets, res = run(sc)
    cells, overlap = ovs.ovs_grid_check(scene.ctx.ctx, 1)
    assert 0 < cells[2] <= 8 and overlap
    assert sum(cells) == donor.n_cells
    assert check(sc, fsets, res) > 10000


def test_double_wrapped_annulus_needs_the_caller_flag(torch_cuda):
    na, nr, nz = 24, 6, 4
    th = 4.0 * np.pi * np.arange(na) / na  # the azimuth goes round twice: every point lies in two cells
    r = np.linspace(1.0, 2.0, nr)
    z = np.linspace(0.0, 1.0, nz)
    T, Rr, Z = np.meshgrid(th, r, z, indexing="ij")
    flat = lambda a: np.ascontiguousarray(a.transpose(2, 1, 0).ravel())
    donor = gen.Grid("annulus", (na, nr, nz), (True, False, False), flat(Rr * np.cos(T)), flat(Rr * np.sin(T)),
                     flat(Z), 1)
    recv = gen.cartesian_grid("r", (33, 33, 6), (-2.0, -2.0, 0.05), (2.0, 2.0, 0.95), role=0)
    rad = np.hypot(recv.x, recv.y)
    ids = np.nonzero((rad > 1.05) & (rad < 1.95))[0]
    sc = scenario(donor, recv, ids, 6)
    scene, fsets, res = run(sc)
    cells, overlap = ovs.ovs_grid_check(scene.ctx.ctx, 1)
    assert cells[2] == 0 and not overlap and (cells[0] == 0 or cells[1] == 0)  # nothing folded: not detectable
    scene2, fsets2, res2 = run(sc, overlap=True)
    assert ovs.ovs_grid_check(scene2.ctx.ctx, 1)[1]
    assert check(sc, fsets2, res2) > 1000
    # for the record: how many donors the walk alone would have taken from the higher of the two cells
    print("donors differing without the flag:", int(np.sum(res["cell"] != res2["cell"])), "of", len(ids))
