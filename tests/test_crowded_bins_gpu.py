"""Crowded control cells, on the GPU against the oracle.

Around a fish O-grid's tail and head tips the cells converge and thin out, and a control cell (a bin of about
0.6 mean cell extents) lists hundreds to thousands of cells.  ovs_create_grid splits such a control cell into
4 x 4 x 4 finer bins, and the exhaustive search of a point reads only its finer bin's list.  Receiver boxes of
Cartesian nodes are placed over both tips.  With a walk limit of one step from the control cell, nearly every
point goes through the exhaustive search.  The points are found in the grid, or left as orphans inside the body
and in the uncovered tip caps.  Donors are compared with the oracle bit for bit, weights and fields with the
FP32 tolerances of tests/harness.py.
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


def tip_boxes(fish, half=(0.035, 0.035, 0.02), n=(28, 28, 16)):
    """Cartesian receiver grids over the head and tail tips: centred on the innermost ring of the first and
    last polar rows, moved 0.02 body lengths toward the body's middle."""
    na, npol, nr = fish.dims
    P = fish.xyz().reshape(nr, npol, na, 3)  # [k][j][i], i fastest
    boxes = []
    for name, ring in (("tail", P[0, -1]), ("head", P[0, 0])):
        c = ring.mean(axis=0)
        c[0] -= 0.02 * np.sign(c[0])
        boxes.append(gen.cartesian_grid(name, n, c - np.asarray(half), c + np.asarray(half), role=0))
    return boxes


def scenario():
    fish = gen.fish_ogrid("fish", 64, 32, 32, 0.7)
    grids = [fish] + tip_boxes(fish)
    fields = gen.make_fields(np.random.default_rng(11), grids, np.float32)
    sets = [gen.FringeSet(r, np.arange(grids[r].n_nodes, dtype=np.int32), [0], "box->fish") for r in (1, 2)]
    ident = [gen.Motion.identity() for _ in grids]
    return gen.Scenario("crowded", grids, fields, np.float32, dt=1.0, nsteps=1, motion_fn=lambda s: ident,
                        sets_fn=lambda s, m: sets)


def test_crowded_control_cells_are_split_and_searched_exactly(torch_cuda):
    sc = scenario()
    m = sc.motion(0)
    fsets = sc.fringe_sets(0, m)
    n = sum(len(s.node_ids) for s in fsets)
    # FP32 local coordinates and fields, as in the large workloads (with FP64 ones the weights of the thinnest
    # tip cells, whose Jacobians are far from uniform, differed from the oracle's by 1.03e-12 against 1e-12)
    scene = GpuScene(sc, max_points=n, xi_dtype=ovs.OVS_F32)
    nbins, nreg, ncrowd, nsub = ovs.ovs_grid_bins(scene.ctx.ctx, scene.ids[0])
    assert nbins > 0 and nreg >= 61504  # every cell listed at least once
    assert ncrowd > 0 and nsub > 0, (nbins, nreg, ncrowd, nsub)  # the tips crowd some control cells
    scene.ctx.set_options(guess=ovs.OVS_GUESS_BINS, max_walk=1, collect_stats=1)
    scene.ctx.stats(reset=True)
    _, d, out = scene.step(m, fsets)
    st = scene.ctx.stats(reset=True)
    res = GpuScene.to_numpy(d, out)
    oref, frames = OracleScene(sc).step(m, fsets)
    found = 0
    for k, (s, part, (od, oq)) in enumerate(zip(fsets, split(res, [len(s.node_ids) for s in fsets]), oref)):
        found += compare(part, od, oq, sc, frames, s.receiver, ovs.OVS_F32, label=f"crowded set {k}")
    assert found > 1000 and n - found > 1000  # both donors and orphans near the tips
    assert st["fallback"] > n // 4, st  # many points took the exhaustive search
