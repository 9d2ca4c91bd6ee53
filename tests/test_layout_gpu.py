"""Field layouts of ovs_interpolate: four arrays, one array of (u, v, w, p) records per node, strided rows and
records that are not 16-byte aligned all give the same bits (the same products summed in the same order)."""
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


@pytest.mark.parametrize("cfg", [0, 1])
def test_field_layouts_equal(torch_cuda, cfg):
    t = torch_cuda
    sc = gen.config(cfg)
    m = sc.motion(0)
    fsets = sc.fringe_sets(0, m)
    n = sum(len(s.node_ids) for s in fsets)
    scene = GpuScene(sc, max_points=n + 1024)
    _, d, _ = scene.step(m, fsets)
    sets = scene.upload_sets(fsets)
    ref = [o.clone() for o in scene.ctx.interpolate(sets, d, scene.fields)]
    dev = scene.ctx.device
    for layout in ("records", "rows of 5", "unaligned records"):
        fl = []
        for f in scene.fields:
            A = t.stack(f, 1)  # (nodes, 4)
            if layout == "records":
                fl.append(A.contiguous())
            elif layout == "rows of 5":
                B = t.full((A.shape[0], 5), float("nan"), dtype=A.dtype, device=dev)
                B[:, :4] = A
                fl.append(B)
            else:
                buf = t.empty(A.numel() + 1, dtype=A.dtype, device=dev)
                V = buf[1:].view(A.shape[0], 4)  # 4 or 8 bytes past a 16-byte boundary
                V.copy_(A)
                fl.append(V)
        out = scene.ctx.interpolate(sets, d, fl)
        scene.ctx.sync()
        for c in range(4):
            a, b = out[c].cpu().numpy(), ref[c].cpu().numpy()
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), (layout, c)
    assert n > 10_000
