"""Shared helpers of the GPU parity tests: run a scenario through libovs (C ABI via the thin binding) and
through the oracle on the same seeded inputs, and compare element by element.

Tolerances (written here, used by every parity test):
  donors        grid id, cell id and status (low 4 bits) bit-exact
  weights       max over the 8 trilinear weights |w - w_ref| <= 1e-12 (FP64 xi) / 1e-5 (FP32 xi)
  fields        |q - q_ref| <= tol * scale, tol = 1e-11 (FP64 fields) / 1e-5 (FP32 fields), where scale is the
                largest |value| of the donor's 8 nodes plus the frame-velocity magnitudes |V| + |omega||r| of both
                frames (the terms the velocity transform adds)
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1910_09315_gb300 import ovs

W_TOL = {ovs.OVS_F64: 1e-12, ovs.OVS_F32: 1e-5}
F_TOL = {np.float64: 1e-11, np.float32: 1e-5}


def weights(xi: np.ndarray) -> np.ndarray:
    """(n,3) -> (n,8) trilinear weights, corner a = di + 2dj + 4dk (test-side, for comparing xi)."""
    u, v, w = xi[:, 0:1], xi[:, 1:2], xi[:, 2:3]
    cols = []
    for a in range(8):
        cols.append(((u if a & 1 else 1 - u) * (v if a & 2 else 1 - v) * (w if a & 4 else 1 - w))[:, 0])
    return np.stack(cols, axis=1)


class GpuScene:
    """A gen.Scenario living on the GPU behind libovs."""

    def __init__(self, sc, max_points: int, xi_dtype: int = ovs.OVS_F32, device: int = 0):
        import torch

        self.torch = torch
        self.sc = sc
        self.xi_dtype = xi_dtype
        self.ctx = ovs.Context(device=device, max_points=max_points)
        self.ids = []
        for g in sc.grids:
            self.ids.append(self.ctx.add_grid(g.x, g.y, g.z, g.dims, g.periodic, g.role))
        fdt = torch.float64 if sc.field_dtype == np.float64 else torch.float32
        self.fields = [tuple(torch.as_tensor(f[k]).to(self.ctx.device, fdt) for k in ("u", "v", "w", "p"))
                       for f in sc.fields]

    def set_iblank(self, gid, mask):
        """Blanked nodes of grid gid (uint8 host array, 0 = blanked) or None (every node active)."""
        if not hasattr(self, "_iblank"):
            self._iblank = {}
        if mask is None:
            self._iblank.pop(gid, None)
            ovs.ovs_set_iblank(self.ctx.ctx, self.ids[gid], None)
        else:
            m = self.torch.as_tensor(np.ascontiguousarray(mask, dtype=np.uint8)).to(self.ctx.device)
            self._iblank[gid] = m  # the library reads it on the stream: keep it alive
            ovs.ovs_set_iblank(self.ctx.ctx, self.ids[gid], m.data_ptr())

    def set_motion(self, motions):
        for gid, m in zip(self.ids, motions):
            self.ctx.set_motion(gid, m.R, m.c, m.V, m.omega)

    def upload_sets(self, fsets):
        t = self.torch
        return [(s.receiver, t.as_tensor(s.node_ids).to(self.ctx.device), s.donors) for s in fsets]

    def step(self, motions, fsets, interpolate: bool = True):
        self.set_motion(motions)
        sets = self.upload_sets(fsets)
        d = self.ctx.assemble(sets, xi_dtype=self.xi_dtype)
        out = self.ctx.interpolate(sets, d, self.fields) if interpolate else None
        self.ctx.sync()
        return sets, d, out

    @staticmethod
    def to_numpy(d, out=None):
        n = d["n"]
        res = {"grid": d["grid"].cpu().numpy(), "cell": d["cell"].cpu().numpy(),
               "xi": d["xi"].cpu().numpy().astype(np.float64).reshape(3, n).T.copy(),
               "status": d["status"].cpu().numpy()}
        if out is not None:
            res["q"] = np.stack([o.cpu().numpy().astype(np.float64) for o in out])
        return res


class OracleScene:
    def __init__(self, sc):
        self.sc = sc
        self.grids = [oracle.OracleGrid.from_gen(g) for g in sc.grids]
        self.xyz = [g.xyz() for g in sc.grids]

    def step(self, motions, fsets, mode: str = "relative", sample=None):
        frames = [oracle.frame_of(m) for m in motions]
        res = []
        for k, s in enumerate(fsets):
            ids = s.node_ids if sample is None else s.node_ids[sample[k]]
            d = oracle.assemble(self.grids, frames, self.xyz[s.receiver], s.receiver, ids, s.donors)
            q = oracle.interpolate(d, self.sc.fields, frames, s.receiver, mode=mode)
            res.append((d, q))
        return res, frames


def field_scale(sc, frames, receiver, d):
    """Per-point scale of the field tolerance (see module docstring)."""
    n = d.grid.shape[0]
    scale = np.zeros(n)
    for gd in np.unique(d.grid[d.grid >= 0]):
        q = np.nonzero(d.grid == gd)[0]
        f = sc.fields[gd]
        mx = np.zeros(q.size)
        for k in ("u", "v", "w", "p"):
            mx = np.maximum(mx, np.abs(np.asarray(f[k], float)[d.nodes[q]]).max(axis=1))
        fd, fr = frames[gd], frames[receiver]
        extra = (np.linalg.norm(fd.V) + np.linalg.norm(fr.V) +
                 np.linalg.norm(fd.omega) * np.linalg.norm(d.x_in[q] - fd.c, axis=1) +
                 np.linalg.norm(fr.omega) * np.linalg.norm(d.x_in[q] - fr.c, axis=1))
        scale[q] = mx + extra
    return scale


def compare(gpu: dict, ref, q_ref, sc, frames, receiver, xi_dtype, check_fields=True, label=""):
    """Element-by-element comparison of one set's GPU result (slice) with the oracle."""
    if ref.status.shape[0] == 0:
        assert gpu["status"].shape[0] == 0, f"{label}: empty set produced outputs"
        return 0
    st = gpu["status"] & ovs.OVS_STATUS_MASK
    assert np.array_equal(st, ref.status), f"{label}: status differs at {np.nonzero(st != ref.status)[0][:10]}"
    assert np.array_equal(gpu["grid"], ref.grid), f"{label}: donor grid differs"
    bad = np.nonzero(gpu["cell"] != ref.cell)[0]
    assert bad.size == 0, f"{label}: {bad.size} donor cells differ, first {bad[:10]}: gpu {gpu['cell'][bad[:5]]} " \
                          f"oracle {ref.cell[bad[:5]]}"
    found = ref.status == 0
    if found.any():
        dw = np.abs(weights(gpu["xi"][found]) - ref.w[found]).max()
        assert dw <= W_TOL[xi_dtype], f"{label}: weights differ by {dw}"
    if check_fields:
        scale = field_scale(sc, frames, receiver, ref)
        tol = F_TOL[sc.field_dtype]
        err = np.abs(gpu["q"] - q_ref) / np.maximum(scale, 1e-300)
        err[:, ~found] = np.abs(gpu["q"][:, ~found])  # no donor -> 0
        assert err.max() <= tol, f"{label}: fields differ, max scaled error {err.max()} (tol {tol})"
    return found.sum()


def split(res: dict, sizes):
    out = []
    b = 0
    for n in sizes:
        out.append({k: (v[..., b:b + n] if k == "q" else v[b:b + n]) for k, v in res.items()})
        b += n
    return out
