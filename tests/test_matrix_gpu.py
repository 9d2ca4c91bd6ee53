"""The interpolation matrix (paper Sec. 2.2.6, the boundary interpolation as a sparse matrix) on the GPU:

* its columns are the donor cells' corner nodes (global numbering) and its values the trilinear weights, equal
  to the oracle's (columns exact, weights within the parity tolerance);
* A x with x = every grid's node field reproduces ovs_interpolate without the frame transform;
* rows of points without a donor are empty; an empty call gives row_ptr = [0].
"""
import numpy as np
import pytest

import gen
from harness import W_TOL, GpuScene, OracleScene, split
from paper_1910_09315_gb300 import ovs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def run(sc, xi_dtype):
    m = sc.motion(0)
    fsets = sc.fringe_sets(0, m)
    n = sum(len(s.node_ids) for s in fsets)
    scene = GpuScene(sc, max_points=n + 1024, xi_dtype=xi_dtype)
    scene.ctx.set_options(velocity_mode=ovs.OVS_VEL_NONE)
    _, d, out = scene.step(m, fsets)
    return scene, m, fsets, d, out


@pytest.mark.parametrize("cfg,xi_dtype", [(0, ovs.OVS_F64), (0, ovs.OVS_F32), (1, ovs.OVS_F32)])
def test_matrix_applies_like_interpolate(torch_cuda, cfg, xi_dtype):
    t = torch_cuda
    sc = gen.config(cfg)
    scene, m, fsets, d, out = run(sc, xi_dtype)
    f64 = sc.field_dtype == np.float64
    row_ptr, col, val = scene.ctx.interp_matrix(d, ovs.OVS_F64 if f64 else ovs.OVS_F32)
    scene.ctx.sync()
    rp = row_ptr.cpu().numpy().astype(np.int64)
    st = d["status"].cpu().numpy() & ovs.OVS_STATUS_MASK
    found = (st == ovs.OVS_STATUS_FOUND) & (d["grid"].cpu().numpy() >= 0)
    assert rp[0] == 0 and np.array_equal(np.diff(rp), 8 * found.astype(np.int64))
    assert found.sum() > 0.9 * found.size
    for c in range(4):
        x = t.cat([scene.fields[g][c] for g in range(len(sc.grids))])
        y = scene.ctx.spmv(row_ptr, col, val, x).cpu().numpy().astype(np.float64)
        ref = out[c].cpu().numpy().astype(np.float64)
        scale = 1.0 + np.abs(ref).max()
        tol = 1e-12 if f64 else 1e-6
        assert np.abs(y - ref).max() <= tol * scale, (c, np.abs(y - ref).max())
        assert np.all(y[~found] == 0)


def test_matrix_equals_oracle_weights(torch_cuda):
    sc = gen.config(0)
    scene, m, fsets, d, out = run(sc, ovs.OVS_F64)
    row_ptr, col, val = scene.ctx.interp_matrix(d, ovs.OVS_F64)
    scene.ctx.sync()
    rp = row_ptr.cpu().numpy()
    cols = col.cpu().numpy()
    vals = val.cpu().numpy()
    offsets = np.concatenate([[0], np.cumsum([g.n_nodes for g in sc.grids])])
    oref, _ = OracleScene(sc).step(m, fsets)
    base = 0
    checked = 0
    for s, (od, _) in zip(fsets, oref):
        for q in np.nonzero(od.status == 0)[0]:
            r = base + q
            e0, e1 = rp[r], rp[r + 1]
            assert e1 - e0 == 8
            assert np.array_equal(cols[e0:e1], offsets[od.grid[q]] + od.nodes[q])
            assert np.abs(vals[e0:e1] - od.w[q]).max() <= W_TOL[ovs.OVS_F64]
            checked += 1
        base += len(s.node_ids)
    assert checked > 10_000


def test_matrix_empty_call(torch_cuda):
    t = torch_cuda
    sc = gen.config(0)
    scene = GpuScene(sc, max_points=1024)
    d = scene.ctx.alloc_donors(0)
    row_ptr, col, val = scene.ctx.interp_matrix(d)
    y = scene.ctx.spmv(row_ptr, col, val, t.zeros(1, dtype=t.float32, device=scene.ctx.device))
    scene.ctx.sync()
    assert row_ptr.cpu().tolist() == [0] and y.numel() == 0
