"""ovs_assemble_noalloc: the assembly entry point for callers that cannot allocate device memory when they
call it (solver plug-ins whose host application owns all device memory, time loops that must not take the
implicit synchronisation of cudaMalloc/cudaFree in the middle of a step).  It keeps its slow-path queue in a
fixed array inside the library; these tests call it through the C ABI and check it against ovs_assemble, in
every guess mode (previous donor, control cell, a trained guess network), on two calls in a row, and that a
warm call leaves the device's free memory unchanged.

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


def noalloc(scene, sets, d):
    """Call ovs_assemble_noalloc through the C ABI into the caller's output arrays d."""
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


def train_body_network(scene, sc, gid=1):
    """A small guess network for body grid gid, trained by the library on samples of the grid itself."""
    cells, xi = gen.mlp_training_samples(1, sc.grids[gid], 200_000)
    rng = np.random.default_rng(5)
    H = 32
    init = np.concatenate([rng.normal(0, 0.8, 3 * H), np.zeros(H), rng.normal(0, 1 / np.sqrt(H), H * H),
                           np.zeros(H), rng.normal(0, 1 / np.sqrt(H), 3 * H), np.zeros(3)]).astype(np.float32)
    scene.ctx.train_guess(gid, cells, xi.astype(np.float32), init, hidden=H, epochs=8, batch=8192, lr=3e-3)


GUESS = {"hint": ovs.OVS_GUESS_HINT, "bins": ovs.OVS_GUESS_BINS, "mlp": ovs.OVS_GUESS_MLP}


@pytest.mark.parametrize("cfg,step,xi_dtype,guess", [(0, 0, ovs.OVS_F64, "hint"), (1, 3, ovs.OVS_F32, "hint"),
                                                      (1, 3, ovs.OVS_F32, "bins"), (1, 3, ovs.OVS_F32, "mlp")])
def test_noalloc_matches_assemble_twice(torch_cuda, cfg, step, xi_dtype, guess):
    sc = gen.config(cfg)
    m = sc.motion(step)
    fsets = sc.fringe_sets(step, m)
    n = sum(len(s.node_ids) for s in fsets)
    scene = GpuScene(sc, max_points=n, xi_dtype=xi_dtype)
    if guess == "mlp":
        train_body_network(scene, sc)
    scene.ctx.set_options(guess=GUESS[guess], collect_stats=1)
    scene.set_motion(m)
    sets = scene.upload_sets(fsets)
    # every call starts from the same (cold) hints, so that each one takes the same start for every point
    ovs.ovs_reset_hints(scene.ctx.ctx)
    scene.ctx.stats(reset=True)
    ref = GpuScene.to_numpy(scene.ctx.assemble(sets, xi_dtype=xi_dtype))
    scene.ctx.sync()
    st_ref = scene.ctx.stats(reset=True)
    outs = [scene.ctx.alloc_donors(n, xi_dtype) for _ in range(2)]  # the caller's outputs, made beforehand
    got, st = [], []
    for k in range(2):  # two calls in a row: the shared array keeps the last call's contents
        ovs.ovs_reset_hints(scene.ctx.ctx)
        free0 = torch_cuda.cuda.mem_get_info(scene.ctx.device)[0]
        got.append(noalloc(scene, sets, outs[k]))
        free1 = torch_cuda.cuda.mem_get_info(scene.ctx.device)[0]
        st.append(scene.ctx.stats(reset=True))
        if k == 1:  # after the first call's one-time set-up, a call takes no device memory
            assert free1 == free0, (free0, free1)
    for g, s in zip(got, st):
        same(ref, g, xi_dtype)
        assert s["points"] == st_ref["points"] == n
        assert s["guess_used"] == st_ref["guess_used"]
    assert (ref["status"] & ovs.OVS_STATUS_MASK == 0).sum() > 20000
    if guess == "mlp":
        assert st_ref["guess_used"] > 10_000  # the learned-guess pass ran in both entry points


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
