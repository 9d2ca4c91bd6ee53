"""Schools of fish (many body grids, body-to-body and multi-donor sets) on the GPU against the oracle.

* 8 fish in a 384x256x128 background: steps 0 and 1 (cold, then warm from the previous donors) on a seeded 20%
  sample of every set, FP32 xi, FP32 fields;
* 16 fish in a 512x384x256 background (~50M nodes): step 0 on a seeded 1% sample of every set;
* the body-to-body sets find their donors in the other body, not in the background.
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


def sampled(fsets, frac, seed):
    rng = np.random.default_rng(seed)
    return [np.sort(rng.choice(len(s.node_ids), size=max(1, int(len(s.node_ids) * frac)), replace=False))
            for s in fsets]


def check_step(sc, scene, ref, step, frac, seed, label, fused=False):
    m = sc.motion(step)
    fsets = sc.fringe_sets(step, m)
    if fused:  # ovs_assemble_interpolate: one pass per point
        scene.set_motion(m)
        d, out = scene.ctx.assemble_interpolate(scene.upload_sets(fsets), scene.fields, xi_dtype=scene.xi_dtype)
        scene.ctx.sync()
    else:
        _, d, out = scene.step(m, fsets)
    res = GpuScene.to_numpy(d, out)
    parts = split(res, [len(s.node_ids) for s in fsets])
    sample = sampled(fsets, frac, seed)
    oref, frames = ref.step(m, fsets, sample=sample)
    total = 0
    for k, (s, part, (od, oq)) in enumerate(zip(fsets, parts, oref)):
        part = {kk: (v[..., sample[k]] if kk == "q" else v[sample[k]]) for kk, v in part.items()}
        total += compare(part, od, oq, sc, frames, s.receiver, ovs.OVS_F32, label=f"{label} set {k} ({s.kind})")
    return fsets, parts, total


def body_to_body_found_in_body(fsets, parts):
    hits = 0
    for s, part in zip(fsets, parts):
        if s.kind != "body->body":
            continue
        found = (part["status"] & ovs.OVS_STATUS_MASK) == ovs.OVS_STATUS_FOUND
        hits += int(np.sum(found & (part["grid"] == s.donors[0])))
    return hits


def test_school_of_8(torch_cuda):
    sc = gen.config(3)
    n = max(sum(len(s.node_ids) for s in sc.fringe_sets(t)) for t in (0, 1))
    scene = GpuScene(sc, max_points=n + 1024)
    ref = OracleScene(sc)
    checked = 0
    for step in (0, 1):
        fsets, parts, total = check_step(sc, scene, ref, step, 0.2, 100 + step, f"school8 step {step}")
        checked += total
        assert any(s.kind == "body->body" for s in fsets)
        assert any(s.receiver == 0 and len(s.donors) > 1 for s in fsets)
        assert body_to_body_found_in_body(fsets, parts) > 0
    assert checked > 200_000


def test_school_of_8_fused_call(torch_cuda):
    """The step as the bench runs it: donors and fields from ovs_assemble_interpolate, cold then warm."""
    sc = gen.config(3)
    n = max(sum(len(s.node_ids) for s in sc.fringe_sets(t)) for t in (2, 3))
    scene = GpuScene(sc, max_points=n + 1024)
    ref = OracleScene(sc)
    checked = 0
    for step in (2, 3):
        fsets, parts, total = check_step(sc, scene, ref, step, 0.1, 200 + step, f"school8 fused step {step}",
                                         fused=True)
        checked += total
        assert body_to_body_found_in_body(fsets, parts) > 0
    assert checked > 100_000


@pytest.mark.slow
def test_school_of_16_sampled(torch_cuda):
    sc = gen.config(4)
    m = sc.motion(0)
    n = sum(len(s.node_ids) for s in sc.fringe_sets(0, m))
    scene = GpuScene(sc, max_points=n + 1024)
    fsets, parts, total = check_step(sc, scene, OracleScene(sc), 0, 0.01, 7, "school16 step 0", fused=True)
    assert len(fsets) > 32
    assert total > 20_000
    assert body_to_body_found_in_body(fsets, parts) > 0
