"""Checkpoint / resume (ovs_get_donors / ovs_set_donors): the previous donors are the whole state a time loop
carries between steps (with the guess networks, which have their own export), so a run stopped after two
steps and resumed in a fresh context from the exported donors gives the uninterrupted run's next donors bit
for bit; imported garbage never changes a donor, only where the search starts."""
import numpy as np
import pytest

import gen
from harness import GpuScene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def donors_bits(d):
    out = {k: d[k].cpu().numpy().copy() for k in ("grid", "cell", "status")}
    out["xi"] = d["xi"].cpu().numpy().view(np.uint32 if d["xi"].element_size() == 4 else np.uint64).copy()
    return out


def test_resume_gives_the_uninterrupted_donors(torch_cuda):
    t = torch_cuda
    sc = gen.config(1)
    steps = []
    for s in range(4):
        m = sc.motion(s)
        steps.append((m, sc.fringe_sets(s, m)))
    n = max(sum(len(x.node_ids) for x in fs) for _, fs in steps)
    # the uninterrupted run
    a = GpuScene(sc, max_points=n + 1024)
    for m, fs in steps[:3]:
        a.step(m, fs, interpolate=False)
    _, d, _ = a.step(*steps[3], interpolate=False)
    want = donors_bits(d)
    # stopped after two steps, its donors exported
    b = GpuScene(sc, max_points=n + 1024)
    for m, fs in steps[:2]:
        b.step(m, fs, interpolate=False)
    saved = [b.ctx.get_donors(g) for g in range(len(sc.grids))]
    b.ctx.sync()
    assert any(int((x != -1).sum()) > 1000 for x in saved)
    # resumed in a fresh context
    c = GpuScene(sc, max_points=n + 1024)
    for g, x in enumerate(saved):
        c.ctx.set_donors(g, x)
    c.ctx.sync()
    c.step(*steps[2], interpolate=False)
    _, d, _ = c.step(*steps[3], interpolate=False)
    got = donors_bits(d)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
    # garbage imported as previous donors changes no donor (only the masked status bits may differ)
    e = GpuScene(sc, max_points=n + 1024)
    rng = np.random.default_rng(1)
    for g in range(len(sc.grids)):
        junk = rng.integers(-2**31, 2**31 - 1, size=sc.grids[g].n_nodes, dtype=np.int64).astype(np.int32)
        e.ctx.set_donors(g, t.as_tensor(junk).to(e.ctx.device))
        e.ctx.sync()
    _, d, _ = e.step(*steps[3], interpolate=False)
    got = donors_bits(d)
    import paper_1910_09315_gb300.ovs as ovs

    for k in ("grid", "cell"):
        assert np.array_equal(got[k], want[k]), k
    assert np.array_equal(got["status"] & ovs.OVS_STATUS_MASK, want["status"] & ovs.OVS_STATUS_MASK)
