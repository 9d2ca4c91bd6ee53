"""ovs_assemble_noalloc: the assembly entry point for callers that cannot allocate device memory when they
call it (code running under CUDA stream capture, solver plug-ins whose host owns all device memory, time
loops that must not take cudaMalloc's implicit synchronisation).  It keeps its slow-path queue in a fixed
array inside the library; these tests call it through the C ABI and check it against ovs_assemble.

Collected last on purpose (file name), so a run that stops at the first failure has run everything else.
Works alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import gen
from harness import W_TOL, GpuScene, weights
from paper_1910_09315_gb300 import ovs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def noalloc(scene, sets, xi_dtype):
    """Call ovs_assemble_noalloc through the C ABI into fresh output arrays."""
    n = sum(int(s[1].numel()) for s in sets)
    d = scene.ctx.alloc_donors(n, xi_dtype)  # outputs are the caller's; the entry point allocates nothing
    arr = ovs.make_sets(sets)
    rc = ovs.load().ovs_assemble_noalloc(scene.ctx.ctx, arr, len(sets), ctypes.byref(scene.ctx.donors_struct(d)))
    assert rc == ovs.OVS_OK, ovs.ovs_last_error(scene.ctx.ctx)
    scene.ctx.sync()
    return GpuScene.to_numpy(d)


def same(a, b, xi_dtype):
    assert np.array_equal(a["grid"], b["grid"])
    assert np.array_equal(a["cell"], b["cell"])
    assert np.array_equal(a["status"] & ovs.OVS_STATUS_MASK, b["status"] & ovs.OVS_STATUS_MASK)
    found = (a["status"] & ovs.OVS_STATUS_MASK) == ovs.OVS_STATUS_FOUND
    if found.any():
        assert np.abs(weights(a["xi"][found]) - weights(b["xi"][found])).max() <= W_TOL[xi_dtype]


@pytest.mark.parametrize("cfg,step,xi_dtype", [(0, 0, ovs.OVS_F64), (1, 3, ovs.OVS_F32)])
def test_noalloc_matches_assemble_twice(torch_cuda, cfg, step, xi_dtype):
    sc = gen.config(cfg)
    m = sc.motion(step)
    fsets = sc.fringe_sets(step, m)
    scene = GpuScene(sc, max_points=sum(len(s.node_ids) for s in fsets), xi_dtype=xi_dtype)
    scene.set_motion(m)
    sets = scene.upload_sets(fsets)
    ref = GpuScene.to_numpy(scene.ctx.assemble(sets, xi_dtype=xi_dtype))
    scene.ctx.sync()
    first = noalloc(scene, sets, xi_dtype)
    second = noalloc(scene, sets, xi_dtype)  # the shared array keeps the last call's contents
    same(ref, first, xi_dtype)
    same(ref, second, xi_dtype)
    assert (ref["status"] & ovs.OVS_STATUS_MASK == 0).sum() > 20000


def test_noalloc_rejects_more_than_its_capacity(torch_cuda):
    sc = gen.config(0)
    scene = GpuScene(sc, max_points=16)
    n = ovs.OVS_NOALLOC_MAX_POINTS + 1
    ids = torch_cuda.zeros(n, dtype=torch_cuda.int32, device=scene.ctx.device)
    d = scene.ctx.alloc_donors(n, ovs.OVS_F32)
    rc = ovs.load().ovs_assemble_noalloc(scene.ctx.ctx, ovs.make_sets([(0, ids, [1])]), 1,
                                         ctypes.byref(scene.ctx.donors_struct(d)))
    assert rc == ovs.OVS_ERR_WORKSPACE
    assert "fixed capacity" in ovs.ovs_last_error(scene.ctx.ctx)
    scene.ctx.sync()
