"""The learned initial guess on the GPU, against the FP64 oracle.

* the training kernel's loss and gradients (FP32) equal the oracle's FP64 analytic ones (which are pinned to
  finite differences in test_oracle_pins.py);
* the tensor-core inference (FP16 operands, FP32 accumulation, layer 1 and W3 split into hi/lo halves) equals
  the oracle's forward pass evaluated with the same FP16 roundings;
* one Adam step equals the oracle's;
* a network trained on the O-grid's own samples makes the search cheaper where there is no previous donor
  (cold start), leaves every donor bit-identical, and the warm-step comparison is reported, not hidden.
"""
import numpy as np
import pytest

import gen
import oracle
from harness import GpuScene
from paper_1910_09315_gb300 import ovs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def random_params(rng, H):
    return {"W1": rng.normal(0, 0.8, (H, 3)), "b1": rng.normal(0, 0.1, H), "W2": rng.normal(0, 1.0 / np.sqrt(H), (H, H)),
            "b2": rng.normal(0, 0.1, H), "W3": rng.normal(0, 1.0 / np.sqrt(H), (3, H)), "b3": rng.normal(0, 0.1, 3)}


def flat(P):
    return np.concatenate([P["W1"].ravel(), P["b1"], P["W2"].ravel(), P["b2"], P["W3"].ravel(), P["b3"]])


def unflat(v, H):
    o = 0
    P = {}
    for k, shape in (("W1", (H, 3)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (3, H)), ("b3", (3,))):
        n = int(np.prod(shape))
        P[k] = v[o:o + n].reshape(shape)
        o += n
    return P


def f16(x):
    """Round to IEEE binary16 (nearest, ties to even), returned as float64."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def small_scene(torch_cuda):
    sc = gen.config(0)
    return GpuScene(sc, max_points=1024)


@pytest.mark.parametrize("H", [32, 64, 128])
def test_training_gradients_match_oracle(torch_cuda, H):
    t = torch_cuda
    rng = np.random.default_rng(20 + H)
    P = random_params(rng, H)
    n = 300
    x = rng.uniform(-1, 1, (n, 3))
    y = rng.uniform(0, 1, (n, 3))
    L, G = oracle.mlp_loss_grads(P, x, y)
    scene = small_scene(t)
    dev = scene.ctx.device
    xs = t.as_tensor(x.T.copy().ravel(), dtype=t.float32, device=dev)
    ts = t.as_tensor(y.T.copy().ravel(), dtype=t.float32, device=dev)
    ps = t.as_tensor(flat(P), dtype=t.float32, device=dev)
    # the oracle at the FP32-rounded parameters and data the kernel sees
    L, G = oracle.mlp_loss_grads(unflat(ps.cpu().double().numpy(), H), xs.cpu().double().numpy().reshape(3, n).T,
                                 ts.cpu().double().numpy().reshape(3, n).T)
    grads = t.zeros(ovs.ovs_guess_param_count(H), dtype=t.float32, device=dev)
    loss = t.zeros(1, dtype=t.float32, device=dev)
    ovs.ovs_mlp_loss_grad(scene.ctx.ctx, H, n, xs.data_ptr(), ts.data_ptr(), ps.data_ptr(), grads.data_ptr(),
                          loss.data_ptr())
    scene.ctx.sync()
    assert float(loss.cpu()) == pytest.approx(L, rel=1e-5)
    ref = flat(G)
    got = grads.cpu().double().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-4 * scale, (np.abs(got - ref).max(), scale)


@pytest.mark.parametrize("H", [32, 64, 128])
def test_tensor_core_inference_matches_oracle(torch_cuda, H):
    t = torch_cuda
    rng = np.random.default_rng(40 + H)
    P = random_params(rng, H)
    scene = small_scene(t)
    dev = scene.ctx.device
    ps = t.as_tensor(flat(P), dtype=t.float32, device=dev)
    ovs.ovs_guess_set_params(scene.ctx.ctx, 1, H, ps.data_ptr())
    n = 1000 + 7  # ragged tail: not a multiple of the 16-point tile
    x = rng.uniform(-1, 1, (n, 3))
    xs = t.as_tensor(x.T.copy().ravel(), dtype=t.float32, device=dev)
    out = t.empty(3 * n, dtype=t.float32, device=dev)
    ovs.ovs_guess_eval(scene.ctx.ctx, 1, n, xs.data_ptr(), out.data_ptr())
    scene.ctx.sync()
    got = out.cpu().double().numpy().reshape(3, n).T
    # reference: FP32 parameters; layer 1 exact (its FP16 hi/lo splits reach about FP32); the activations of
    # both hidden layers and W2 rounded to FP16; W3 exact (hi/lo split); FP64 elsewhere
    Pf = unflat(ps.cpu().double().numpy(), H)
    xf = xs.cpu().double().numpy().reshape(3, n).T
    h1 = f16(oracle.silu(xf @ Pf["W1"].T + Pf["b1"]))
    h2 = f16(oracle.silu(h1 @ f16(Pf["W2"]).T + Pf["b2"]))
    ref = h2 @ Pf["W3"].T + Pf["b3"]
    assert np.abs(got - ref).max() <= 5e-3 * (1 + np.abs(ref).max())
    # and close to the plain FP64 network (FP16 roundings are the only difference)
    ref64, _ = oracle.mlp_forward(Pf, xf)
    assert np.abs(got - ref64).max() <= 0.05 * (1 + np.abs(ref64).max())


def test_adam_step_matches_oracle(torch_cuda):
    """One training step of ovs_train_guess (gradient + Adam) on one batch equals the oracle's Adam step."""
    t = torch_cuda
    H = 32
    sc = gen.config(0)
    scene = GpuScene(sc, max_points=1024)
    rng = np.random.default_rng(5)
    P = random_params(rng, H)
    g = sc.grids[1]
    cells, xi = gen.mlp_training_samples(0, g, 256)
    init = flat(P)
    loss = scene.ctx.train_guess(1, cells, xi.astype(np.float32), init.astype(np.float32), hidden=H, epochs=1,
                                 batch=256, lr=1e-3)
    got = t.empty(ovs.ovs_guess_param_count(H), dtype=t.float32, device=scene.ctx.device)
    assert ovs.ovs_guess_get_params(scene.ctx.ctx, 1, got.data_ptr()) == H
    scene.ctx.sync()
    # oracle: inputs/targets from the grid (FP64 trilinear map), MSE gradient, one Adam step
    og = oracle.OracleGrid.from_gen(g)
    xyz = g.xyz()
    X = np.zeros((256, 3))
    T = np.zeros((256, 3))
    ci, cj = og.cell_dims[0], og.cell_dims[1]
    lo = xyz.min(0) - 4e-6 * (xyz.max(0) - xyz.min(0)).max()
    hi = xyz.max(0) + 4e-6 * (xyz.max(0) - xyz.min(0)).max()
    centre = (0.5 * (lo + hi)).astype(np.float32).astype(np.float64)
    inv_half = (2.0 / (hi - lo)).astype(np.float32).astype(np.float64)
    for q in range(256):
        nodes = og.cell_nodes(cells[q])
        w = oracle.shape(xi[q].astype(np.float32).astype(np.float64))
        p = w @ xyz[nodes]
        X[q] = (p - centre) * inv_half
        c = cells[q]
        ijk = (c % ci, (c // ci) % cj, c // (ci * cj))
        T[q] = (np.array(ijk) + xi[q].astype(np.float32)) / np.array(og.cell_dims)
    P32 = unflat(init.astype(np.float32).astype(np.float64), H)
    L, G = oracle.mlp_loss_grads(P32, X, T)
    m = {k: np.zeros_like(v) for k, v in P32.items()}
    v = {k: np.zeros_like(v) for k, v in P32.items()}
    oracle.adam_step(P32, G, m, v, 1, lr=1e-3)
    assert loss == pytest.approx(L, rel=1e-3)
    # Adam's first step is lr * g / (|g| + 1e-8): compare where the gradient is not at FP32 noise level
    gref = np.abs(flat(G))
    sel = gref > 1e-4 * gref.max()
    assert sel.sum() > 0.5 * sel.size
    assert np.abs(got.cpu().double().numpy() - flat(P32))[sel].max() <= 2e-5


def test_trained_guess_gains_on_cold_start(torch_cuda):
    """Train the O-grid's network (64 wide) on samples of the grid itself; with no previous donor, starting
    the walk from the network's cell takes fewer walk steps than starting from the control cell, and every donor
    is the same bit for bit."""
    t = torch_cuda
    sc = gen.config(1)
    scene = GpuScene(sc, max_points=800_000)
    body = sc.grids[1]
    cells, xi = gen.mlp_training_samples(1, body, 1_000_000)
    rng = np.random.default_rng(1)
    init = flat(random_params(rng, 64)).astype(np.float32)
    loss = scene.ctx.train_guess(1, cells, xi.astype(np.float32), init, hidden=64, epochs=60, batch=8192, lr=3e-3,
                                 lr_final=1e-5)
    print("final training loss", loss)
    assert loss < 3e-3  # mean squared error of normalised curvilinear coordinates (about 0.1 at the start)
    m = sc.motion(0)
    fsets = sc.fringe_sets(0, m)
    res = {}
    for name, mode in (("bins", ovs.OVS_GUESS_BINS), ("mlp", ovs.OVS_GUESS_MLP_ONLY)):
        ovs.ovs_reset_hints(scene.ctx.ctx)
        scene.ctx.set_options(guess=mode, collect_stats=1)
        scene.ctx.stats(reset=True)
        _, d, _ = scene.step(m, fsets, interpolate=False)
        res[name] = (GpuScene.to_numpy(d), scene.ctx.stats(reset=True))
    (a, sa), (b, sb) = res["bins"], res["mlp"]
    assert np.array_equal(a["cell"], b["cell"]) and np.array_equal(a["grid"], b["grid"])
    assert np.array_equal(a["status"] & 15, b["status"] & 15)
    print("cold start walk steps: control cell", sa["walk_steps"], "network", sb["walk_steps"], "network guesses",
          sb["guess_used"])
    assert sb["guess_used"] > 600_000
    assert sb["walk_steps"] < sa["walk_steps"]


def test_school_learned_guess_in_the_fused_call(torch_cuda):
    """Eight fish with networks of two widths (32 on even fish, 128 on odd ones, so one call runs both tile codes
    and a warp can meet two networks at a set boundary): the learned start, cold (network for every point that
    has no previous donor) and warm, gives the plain start's donors bit for bit and its fields to within the
    parity tolerance (a different start can leave the FP32 local coordinates different in their last bits)."""
    from harness import F_TOL, W_TOL, weights

    sc = gen.config(3)
    m0 = sc.motion(4)
    f0 = sc.fringe_sets(4, m0)
    n = sum(len(s.node_ids) for s in f0) + 1024
    plain = GpuScene(sc, max_points=n)
    learned = GpuScene(sc, max_points=n)
    rng = np.random.default_rng(3)
    bodies = [gi for gi, g in enumerate(sc.grids) if g.role == 1]
    for gi in bodies:
        H = 32 if gi % 2 == 0 else 128
        cells, xi = gen.mlp_training_samples(3, sc.grids[gi], 200_000)
        learned.ctx.train_guess(gi, cells, xi.astype(np.float32), flat(random_params(rng, H)).astype(np.float32),
                                hidden=H, epochs=6, batch=8192, lr=3e-3)
    plain.ctx.set_options(guess=ovs.OVS_GUESS_HINT)
    learned.ctx.set_options(guess=ovs.OVS_GUESS_MLP, collect_stats=1)

    def fused(scene, m, fs):
        scene.set_motion(m)
        d, out = scene.ctx.assemble_interpolate(scene.upload_sets(fs), scene.fields)
        scene.ctx.sync()
        return GpuScene.to_numpy(d, out)

    used = 0
    for step in (4, 5, 6):  # cold, then warm twice
        m, fs = sc.motion(step), sc.fringe_sets(step)
        a, b = fused(plain, m, fs), fused(learned, m, fs)
        assert np.array_equal(a["grid"], b["grid"]) and np.array_equal(a["cell"], b["cell"]), step
        assert np.array_equal(a["status"] & 15, b["status"] & 15), step
        found = (a["status"] & 15) == 0
        assert np.abs(weights(a["xi"][found]) - weights(b["xi"][found])).max() <= W_TOL[ovs.OVS_F32]
        scale = np.maximum(np.abs(a["q"]), 1.0)
        assert (np.abs(a["q"] - b["q"]) / scale).max() <= 10 * F_TOL[np.float32], step
        used += learned.ctx.stats(reset=True)["guess_used"]
    assert used > 50_000
