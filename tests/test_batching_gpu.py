"""Batching on the GPU: one persistent launch over all sets of all grids, a CUDA graph per kind of call, and the
autotuner's launch shapes.  None of them may change a result: every output equals, bit for bit, that of direct
launches with the default shapes, step after step while the sets change size (and the oracle checks the
direct path in test_parity_gpu.py and test_school_gpu.py)."""
import numpy as np
import pytest

import gen
from harness import GpuScene
from paper_1910_09315_gb300 import ovs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def run(scene, m, fsets):
    _, d, out = scene.step(m, fsets)
    return GpuScene.to_numpy(d, out)


def same(a, b, label):
    for k in a:
        x, y = np.asarray(a[k]), np.asarray(b[k])
        assert x.shape == y.shape, (label, k)
        assert np.array_equal(x, y, equal_nan=True), f"{label}: {k} differs"


@pytest.mark.parametrize("cfg", [1, 3])
def test_graph_equals_direct_over_steps(torch_cuda, cfg):
    sc = gen.config(cfg)
    steps = [0, 1, 2, 7]
    inputs = [(sc.motion(s), sc.fringe_sets(s)) for s in steps]
    sizes = [sum(len(f.node_ids) for f in fs) for _, fs in inputs]
    assert len(set(sizes)) > 1 or cfg == 3  # the sets change size from step to step
    n = max(sizes) + 1024
    direct = GpuScene(sc, max_points=n)
    direct.ctx.set_options(launch=ovs.OVS_LAUNCH_DIRECT)
    graph = GpuScene(sc, max_points=n)
    graph.ctx.set_options(launch=ovs.OVS_LAUNCH_GRAPH)
    for s, (m, fs) in zip(steps, inputs):
        same(run(direct, m, fs), run(graph, m, fs), f"cfg{cfg} step {s}")


def test_autotuned_shapes_keep_results(torch_cuda):
    sc = gen.config(1)
    m0, f0 = sc.motion(0), sc.fringe_sets(0)
    n = max(sum(len(f.node_ids) for f in sc.fringe_sets(s)) for s in (0, 1, 2)) + 1024
    ref = GpuScene(sc, max_points=n)
    ref.ctx.set_options(launch=ovs.OVS_LAUNCH_DIRECT)
    tuned = GpuScene(sc, max_points=n)
    tuned.set_motion(m0)
    best = tuned.ctx.autotune(tuned.upload_sets(f0), tuned.fields, reps=3)
    assert 1 <= best["assemble_blocks_per_sm"] <= 12 and 1 <= best["interp_blocks_per_sm"] <= 32
    assert 1 <= best["slow_blocks_per_sm"] <= 8
    t = ovs.ovs_get_tuning(tuned.ctx.ctx)
    assert t.assemble_blocks_per_sm == best["assemble_blocks_per_sm"]
    # the autotuner's calls ran for real: start both from cold hints again and compare a few steps
    ovs.ovs_reset_hints(tuned.ctx.ctx)
    for s in (0, 1, 2):
        m, fs = sc.motion(s), sc.fringe_sets(s)
        same(run(ref, m, fs), run(tuned, m, fs), f"tuned step {s}")
    # extreme but valid shapes give the same results too
    tuned.ctx.set_tuning(assemble_blocks_per_sm=1, interp_blocks_per_sm=1, slow_blocks_per_sm=8, guess_blocks_per_sm=1)
    ovs.ovs_reset_hints(tuned.ctx.ctx)
    ovs.ovs_reset_hints(ref.ctx.ctx)
    m, fs = sc.motion(3), sc.fringe_sets(3)
    same(run(ref, m, fs), run(tuned, m, fs), "one block per SM")


def test_tuning_is_checked(torch_cuda):
    sc = gen.config(0)
    scene = GpuScene(sc, max_points=1024)
    for bad in ({"assemble_blocks_per_sm": 13}, {"interp_blocks_per_sm": -1}, {"slow_blocks_per_sm": 9},
                {"guess_blocks_per_sm": 33}):
        with pytest.raises(ovs.OvsError):
            scene.ctx.set_tuning(**bad)
    scene.ctx.set_tuning(assemble_blocks_per_sm=0, interp_blocks_per_sm=0, slow_blocks_per_sm=0, guess_blocks_per_sm=0)
    with pytest.raises(ovs.OvsError):
        scene.ctx.set_options(launch=2)
