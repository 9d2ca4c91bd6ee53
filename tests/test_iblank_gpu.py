"""Blanked donors (paper Sec. 2.4: a cell with a blanked corner node never donates) on the GPU against the oracle.

* two overlapping donor grids, the first with randomly blanked nodes: points fall through to the second grid
  or become orphans exactly as the oracle decides (donors bit-exact, weights and fields within tolerance), with
  receivers on nodes, faces and random positions, in FP64 and FP32 xi;
* the 8-fish school with its step's hole cut (background nodes inside a fish body blanked), sampled;
* a cleared mask restores the unmasked donors bit for bit.
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


def run_compare(sc, scene, ref, step, xi_dtype, sample=None, label=""):
    m = sc.motion(step)
    fsets = sc.fringe_sets(step, m)
    _, d, out = scene.step(m, fsets)
    res = GpuScene.to_numpy(d, out)
    parts = split(res, [len(s.node_ids) for s in fsets])
    oref, frames = ref.step(m, fsets, sample=sample)
    total = 0
    for k, (s, part, (od, oq)) in enumerate(zip(fsets, parts, oref)):
        if sample is not None:
            part = {kk: (v[..., sample[k]] if kk == "q" else v[sample[k]]) for kk, v in part.items()}
        total += compare(part, od, oq, sc, frames, s.receiver, xi_dtype, label=f"{label} set {k}")
    return res, total


def overlapping_pair(dtype):
    rng = np.random.default_rng(77)
    a = gen.cartesian_grid("A", (17, 17, 17), (0, 0, 0), (1, 1, 1), role=0)
    # perturb A's interior nodes so that its cells are general hexahedra
    h = 1 / 16
    for arr in (a.x, a.y, a.z):
        arr += 0.2 * h * np.sin(2 * np.pi * a.x + 1.0) * np.sin(2 * np.pi * a.y + 2.0) * np.sin(np.pi * a.z)
    b = gen.cartesian_grid("B", (13, 13, 13), (-0.05, -0.05, -0.05), (1.05, 1.05, 1.05), role=0)
    rec = gen.cartesian_grid("R", (33, 33, 33), (0.01, 0.02, 0.03), (0.99, 0.98, 0.97), role=1)
    ids = np.arange(rec.n_nodes, dtype=np.int32)
    I = gen.Motion.identity()
    fields = gen.make_fields(rng, [a, b, rec], dtype)
    sc = gen.Scenario("overlap", [a, b, rec], fields, dtype, 0.0, 1, lambda s: [I, I, I],
                      lambda s, m: [gen.FringeSet(2, ids, [0, 1], "rec->A,B")])
    mask = (rng.uniform(size=a.n_nodes) > 0.1).astype(np.uint8)
    return sc, mask


@pytest.mark.parametrize("xi_dtype", [ovs.OVS_F64, ovs.OVS_F32])
def test_blanked_cells_fall_through(torch_cuda, xi_dtype):
    sc, mask = overlapping_pair(np.float64 if xi_dtype == ovs.OVS_F64 else np.float32)
    scene = GpuScene(sc, max_points=sc.grids[2].n_nodes + 16, xi_dtype=xi_dtype)
    ref = OracleScene(sc)
    plain, _ = run_compare(sc, scene, ref, 0, xi_dtype, label="unmasked")
    scene.set_iblank(0, mask)
    ref.grids[0].set_iblank(mask)
    masked, n = run_compare(sc, scene, ref, 0, xi_dtype, label="masked")
    moved = np.sum((plain["grid"] == 0) & (masked["grid"] == 1))
    assert moved > 1000 and n > 30_000
    # clearing the mask restores the unmasked answer bit for bit
    scene.set_iblank(0, None)
    ref.grids[0].set_iblank(None)
    again, _ = run_compare(sc, scene, ref, 0, xi_dtype, label="cleared")
    for k in ("grid", "cell"):
        assert np.array_equal(again[k], plain[k])
    # (the status's FALLBACK / REFINED bits record which path decided, which depends on the hints)
    assert np.array_equal(again["status"] & ovs.OVS_STATUS_MASK, plain["status"] & ovs.OVS_STATUS_MASK)


def test_school_hole_cut(torch_cuda):
    sc = gen.config(3)
    m = sc.motion(0)
    fsets = sc.fringe_sets(0, m)
    n = sum(len(s.node_ids) for s in fsets)
    scene = GpuScene(sc, max_points=n + 1024)
    ref = OracleScene(sc)
    masks = sc.meta["iblank_fn"](m)
    for g, mk in enumerate(masks):
        if not np.all(mk):
            scene.set_iblank(g, mk)
            ref.grids[g].set_iblank(mk)
    rng = np.random.default_rng(3)
    sample = [np.sort(rng.choice(len(s.node_ids), size=max(1, len(s.node_ids) // 5), replace=False)) for s in fsets]
    _, total = run_compare(sc, scene, ref, 0, ovs.OVS_F32, sample=sample, label="school hole cut")
    assert total > 100_000
