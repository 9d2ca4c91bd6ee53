"""GPU parity: libovs (through the C ABI) against the FP64 oracle on the same seeded inputs.

Donor grid/cell/status bit-exact; weights and fields within the tolerances of tests/harness.py.  Covers
config 0 in FP64 and FP32, config 1's moving grids over many warm-started steps (full sets, the bench's
workload), config 2 sampled at full size, ties on nodes and faces, ragged and empty sets, orphans,
non-finite inputs, priority lists and the three velocity modes.
"""
import copy

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


def run_and_compare(sc, step, xi_dtype, mode="relative", scene=None, ref=None, sample=None, label=""):
    m = sc.motion(step)
    fsets = sc.fringe_sets(step, m)
    scene = scene or GpuScene(sc, max_points=sum(len(s.node_ids) for s in fsets) + 1024, xi_dtype=xi_dtype)
    vm = {"relative": ovs.OVS_VEL_RELATIVE, "absolute": ovs.OVS_VEL_ABSOLUTE, "none": ovs.OVS_VEL_NONE}[mode]
    scene.ctx.set_options(velocity_mode=vm)
    _, d, out = scene.step(m, fsets)
    res = GpuScene.to_numpy(d, out)
    parts = split(res, [len(s.node_ids) for s in fsets])
    ref = ref or OracleScene(sc)
    oref, frames = ref.step(m, fsets, mode="relative" if mode == "none" else mode, sample=sample)
    total = 0
    for k, (s, part, (od, oq)) in enumerate(zip(fsets, parts, oref)):
        if sample is not None:
            part = {kk: (v[..., sample[k]] if kk == "q" else v[sample[k]]) for kk, v in part.items()}
        if mode == "none":
            # no transform: interpolate u, v, w like p
            frames_id = [oracle.Frame(np.eye(3), np.zeros(3), np.zeros(3), np.zeros(3)) for _ in frames]
            oq = oracle.interpolate(od, sc.fields, frames_id, s.receiver, mode="relative")
            total += compare(part, od, oq, sc, frames_id, s.receiver, xi_dtype, label=f"{label} set {k}")
        else:
            total += compare(part, od, oq, sc, frames, s.receiver, xi_dtype, label=f"{label} set {k}")
    return scene, ref, total


def f32_fields(sc):
    sc2 = copy.copy(sc)
    sc2.fields = [{k: v.astype(np.float32) for k, v in f.items()} for f in sc.fields]
    sc2.field_dtype = np.float32
    return sc2


def test_cfg0_fp64(torch_cuda):
    sc = gen.config(0)
    _, _, n = run_and_compare(sc, 0, ovs.OVS_F64, label="cfg0 f64")
    assert n > 20000


def test_cfg0_mixed_precision(torch_cuda):
    sc = f32_fields(gen.config(0))
    run_and_compare(sc, 0, ovs.OVS_F32, label="cfg0 f32")


@pytest.mark.parametrize("mode", ["absolute", "none"])
def test_cfg0_velocity_modes(torch_cuda, mode):
    sc = gen.config(0)
    run_and_compare(sc, 0, ovs.OVS_F64, mode=mode, label=f"cfg0 {mode}")


def test_cfg1_moving_warm_steps(torch_cuda):
    """The bench's workload: 100 steps of the moving O-grid, hints carried from step to step; full sets
    compared with the oracle at several steps."""
    sc = gen.config(1)
    scene, ref = None, None
    check = {0, 1, 2, 50, 99}
    for step in range(sc.nsteps):
        m = sc.motion(step)
        fsets = sc.fringe_sets(step, m)
        if scene is None:
            scene = GpuScene(sc, max_points=800_000, xi_dtype=ovs.OVS_F32)
        if step in check:
            scene, ref, n = run_and_compare(sc, step, ovs.OVS_F32, scene=scene, ref=ref, label=f"cfg1 step {step}")
            assert n > 600_000
        else:
            scene.step(m, fsets, interpolate=False)


def test_cfg1_cold_equals_warm(torch_cuda):
    sc = gen.config(1)
    m = sc.motion(7)
    fsets = sc.fringe_sets(7, m)
    scene = GpuScene(sc, max_points=800_000, xi_dtype=ovs.OVS_F32)
    scene.step(sc.motion(6), sc.fringe_sets(6), interpolate=False)
    _, dw, _ = scene.step(m, fsets, interpolate=False)
    warm = GpuScene.to_numpy(dw)
    scene.ctx.set_options(guess=ovs.OVS_GUESS_BINS)
    _, dc, _ = scene.step(m, fsets, interpolate=False)
    cold = GpuScene.to_numpy(dc)
    for k in ("grid", "cell"):
        assert np.array_equal(warm[k], cold[k])
    assert np.array_equal(warm["status"] & 15, cold["status"] & 15)
    # deterministic: the same call twice gives bit-identical outputs
    _, dc2, _ = scene.step(m, fsets, interpolate=False)
    again = GpuScene.to_numpy(dc2)
    assert np.array_equal(cold["xi"], again["xi"], equal_nan=True)  # orphans carry NaN local coordinates
    assert np.array_equal(cold["cell"], again["cell"])


def test_cfg2_full_size_sampled(torch_cuda):
    """256^3 background: the whole set on the GPU, a seeded 2% sample checked against the oracle."""
    sc = gen.config(2)
    m = sc.motion(0)
    fsets = sc.fringe_sets(0, m)
    rng = np.random.default_rng(42)
    sample = [np.sort(rng.choice(len(s.node_ids), size=max(1, len(s.node_ids) // 50), replace=False)) for s in fsets]
    run_and_compare(sc, 0, ovs.OVS_F32, sample=sample, label="cfg2 sampled")


# ----------------------------------------------------------------------------- edge cases
def cart(name, n, lo, hi, role):
    return gen.cartesian_grid(name, (n, n, n), (lo,) * 3, (hi,) * 3, role=role)


def mini_scenario(grids, sets_list, motions, dtype=np.float64, seed=5):
    rng = np.random.default_rng(seed)
    fields = gen.make_fields(rng, grids, dtype)
    return gen.Scenario("mini", grids, fields, dtype, 0.0, 1, lambda s: motions, lambda s, m: sets_list)


@pytest.mark.parametrize("xi_dtype", [ovs.OVS_F64, ovs.OVS_F32])
def test_ties_on_nodes_and_faces(torch_cuda, xi_dtype):
    """Receiver nodes exactly on donor nodes, edges and faces: the lowest linear id wins (closed form)."""
    donor = cart("d17", 17, 0.0, 1.0, role=0)
    rec = cart("r33", 33, 0.0, 1.0, role=1)  # every donor node, edge midpoint, face centre and cell centre
    ids = np.arange(rec.n_nodes, dtype=np.int32)
    I = gen.Motion.identity()
    sc = mini_scenario([donor, rec], [gen.FringeSet(1, ids, [0], "ties")], [I, I],
                       dtype=np.float64 if xi_dtype == ovs.OVS_F64 else np.float32)
    _, _, n = run_and_compare(sc, 0, xi_dtype, label="ties")
    assert n == rec.n_nodes
    # closed form of the lowest-id rule on a uniform axis: i* = max(0, ceil(t - 1 - 1e-10)) clamped
    scene = GpuScene(sc, max_points=rec.n_nodes)
    _, d, _ = scene.step([I, I], sc.fringe_sets(0), interpolate=False)
    cell = d["cell"].cpu().numpy()
    t = np.stack([rec.x, rec.y, rec.z], axis=1) * 16
    ijk = np.clip(np.maximum(0, np.ceil(t - 1 - 1e-10)), 0, 15).astype(np.int64)
    expect = ijk[:, 0] + 16 * (ijk[:, 1] + 16 * ijk[:, 2])
    assert np.array_equal(cell, expect)


@pytest.mark.parametrize("xi_dtype", [ovs.OVS_F64, ovs.OVS_F32])
def test_ties_under_a_quarter_turn(torch_cuda, xi_dtype):
    """A moving donor: a Cartesian grid of spacing 1/8 turned a quarter about z and shifted by dyadic offsets, so
    that its frame map is exact in floating point; the receiver's nodes (a lattice of spacing 1/16 over the donor's
    inertial box) land on the donor's nodes, edges, faces and cell centres.  The lowest linear id wins (closed form
    in the donor frame), and the oracle agrees point for point."""
    donor = cart("d9", 9, 0.0, 1.0, role=1)
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])  # body -> inertial: (x, y, z) -> (-y, x, z)
    c = np.array([0.5, 0.25, 0.125])
    rec = gen.cartesian_grid("r17", (17, 17, 17), (-0.5, 0.25, 0.125), (0.5, 1.25, 1.125), role=0)
    ids = np.arange(rec.n_nodes, dtype=np.int32)
    motions = [gen.Motion(R, c, np.array([0.1, 0.0, 0.0]), np.array([0.0, 0.0, 0.7])), gen.Motion.identity()]
    sc = mini_scenario([donor, rec], [gen.FringeSet(1, ids, [0], "ties")], motions,
                       dtype=np.float64 if xi_dtype == ovs.OVS_F64 else np.float32)
    _, _, n = run_and_compare(sc, 0, xi_dtype, label="quarter-turn ties")
    assert n == rec.n_nodes
    scene = GpuScene(sc, max_points=rec.n_nodes, xi_dtype=xi_dtype)
    _, d, _ = scene.step(motions, sc.fringe_sets(0), interpolate=False)
    cell = d["cell"].cpu().numpy()
    xb = np.stack([rec.y - 0.25, 0.5 - rec.x, rec.z - 0.125], axis=1)  # R^T (x - c), exact on these lattices
    t = xb * 8
    ijk = np.clip(np.maximum(0, np.ceil(t - 1 - 1e-10)), 0, 7).astype(np.int64)
    expect = ijk[:, 0] + 8 * (ijk[:, 1] + 8 * ijk[:, 2])
    assert np.array_equal(cell, expect)


def test_ragged_empty_sets_orphans_priority(torch_cuda):
    """Several sets of ragged sizes (0, 1, 31, 33, 257, ...) in one call, an empty set between others, a priority
    list of two donors with fall-through, and points outside every donor (orphans)."""
    g0 = cart("a", 9, 0.0, 1.0, role=0)
    g1 = cart("b", 7, 0.6, 1.8, role=1)
    g2 = gen.cartesian_grid("r", (23, 5, 5), (-0.5, 0.2, 0.3), (2.5, 0.7, 0.8), role=1)
    rng = np.random.default_rng(3)
    R = gen.euler_zyx(0.1, 0.2, 0.3)
    motions = [gen.Motion.identity(), gen.Motion(np.eye(3), np.array([0.05, 0, 0]), np.array([0.1, 0, 0]),
                                                 np.array([0, 0, 0.5])),
               gen.Motion(R, np.array([0.02, -0.01, 0.03]), np.array([0, 0.2, 0]), np.array([0.3, 0, 0]))]
    allr = np.arange(g2.n_nodes, dtype=np.int32)
    sets = []
    for n in (1, 31, 0, 33, 257, g2.n_nodes):
        ids = np.sort(rng.choice(allr, size=min(n, g2.n_nodes), replace=False)).astype(np.int32)
        sets.append(gen.FringeSet(2, ids, [0, 1], f"n{n}"))
    sets.append(gen.FringeSet(0, np.arange(0, g0.n_nodes, 3, dtype=np.int32), [1], "bg->b"))
    sets.append(gen.FringeSet(1, np.arange(g1.n_nodes, dtype=np.int32), [2, 0], "b->r,a"))
    sc = mini_scenario([g0, g1, g2], sets, motions)
    scene, _, n = run_and_compare(sc, 0, ovs.OVS_F64, label="ragged")
    st = GpuScene.to_numpy(scene.ctx.assemble(scene.upload_sets(sets), xi_dtype=ovs.OVS_F64))["status"] & 15
    assert (st == ovs.OVS_STATUS_ORPHAN).sum() > 50 and (st == ovs.OVS_STATUS_FOUND).sum() > 200


def test_nonfinite_inputs_are_badinput(torch_cuda):
    donor = cart("d", 5, 0.0, 1.0, role=0)
    rec = cart("r", 3, 1.0e308, 1.2e308, role=1)  # finite nodes whose inertial image overflows
    motions = [gen.Motion.identity(), gen.Motion(np.eye(3), np.array([1e308, 0, 0]), np.zeros(3), np.zeros(3))]
    sc = mini_scenario([donor, rec], [gen.FringeSet(1, np.arange(27, dtype=np.int32), [0])], motions)
    scene = GpuScene(sc, max_points=64, xi_dtype=ovs.OVS_F64)
    _, d, out = scene.step(motions, sc.fringe_sets(0))
    st = d["status"].cpu().numpy() & 15
    assert np.all(st == ovs.OVS_STATUS_BADINPUT)
    assert np.all(d["cell"].cpu().numpy() == -1)
    assert all(float(o.abs().max()) == 0 for o in out)


def test_argument_errors_do_not_launch(torch_cuda):
    sc = gen.config(0)
    scene = GpuScene(sc, max_points=100)
    fsets = sc.fringe_sets(0)
    with pytest.raises(ovs.OvsError) as e:
        scene.ctx.assemble(scene.upload_sets(fsets))  # more points than the workspace holds
    assert e.value.code == ovs.OVS_ERR_WORKSPACE
    with pytest.raises(ovs.OvsError) as e:
        scene.ctx.set_motion(1, np.diag([1.0, 1.0, -1.0]), np.zeros(3), np.zeros(3), np.zeros(3))
    assert e.value.code == ovs.OVS_ERR_ARG
    bad = [(0, scene.torch.zeros(3, dtype=scene.torch.int32, device=scene.ctx.device), [5])]
    with pytest.raises(ovs.OvsError) as e:
        scene.ctx.assemble(bad)
    assert e.value.code == ovs.OVS_ERR_ARG
    scene.ctx.sync()


# ----------------------------------------------------------------------------- fused assemble + interpolate
def fused_step(scene, motions, fsets):
    scene.set_motion(motions)
    sets = scene.upload_sets(fsets)
    d, out = scene.ctx.assemble_interpolate(sets, scene.fields, xi_dtype=scene.xi_dtype)
    scene.ctx.sync()
    return GpuScene.to_numpy(d, out)


@pytest.mark.parametrize("cfg,xi_dtype", [(0, ovs.OVS_F64), (1, ovs.OVS_F32)])
def test_fused_matches_oracle(torch_cuda, cfg, xi_dtype):
    sc = gen.config(cfg)
    ref = OracleScene(sc)
    steps = [0] if cfg == 0 else [0, 1, 2, 3]
    scene = None
    for step in steps:
        m = sc.motion(step)
        fsets = sc.fringe_sets(step, m)
        scene = scene or GpuScene(sc, max_points=800_000, xi_dtype=xi_dtype)
        res = fused_step(scene, m, fsets)
        parts = split(res, [len(s.node_ids) for s in fsets])
        oref, frames = ref.step(m, fsets)
        for k, (s, part, (od, oq)) in enumerate(zip(fsets, parts, oref)):
            compare(part, od, oq, sc, frames, s.receiver, xi_dtype, label=f"fused cfg{cfg} step {step} set {k}")


def test_fused_equals_separate_calls(torch_cuda):
    sc = gen.config(1)
    m = sc.motion(5)
    fsets = sc.fringe_sets(5, m)
    a = GpuScene(sc, max_points=800_000)
    b = GpuScene(sc, max_points=800_000)
    for step in range(5):  # same warm hints in both contexts
        a.step(sc.motion(step), sc.fringe_sets(step), interpolate=False)
        b.step(sc.motion(step), sc.fringe_sets(step), interpolate=False)
    _, d, out = a.step(m, fsets)
    sep = GpuScene.to_numpy(d, out)
    fus = fused_step(b, m, fsets)
    assert np.array_equal(sep["grid"], fus["grid"]) and np.array_equal(sep["cell"], fus["cell"])
    assert np.array_equal(sep["status"], fus["status"])
    assert np.array_equal(sep["xi"], fus["xi"], equal_nan=True)
    # the same arithmetic on the same inputs, up to the compiler's contraction choices in two different kernels
    assert np.allclose(sep["q"], fus["q"], rtol=1e-6, atol=1e-6)
