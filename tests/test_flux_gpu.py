"""Fluxes at the receivers and the mass-conservation correction on the GPU (ovs_interface_flux) against the oracle.

* face fluxes U = u . S (S = half the cross product of the face diagonals, u = the corners' mean) on a stretched
  curvilinear grid and on the O-grid, whose closed shell surface wraps around its periodic axis; FP64 and FP32
  velocities; several closed surfaces in one call (one of them empty, the others summed in several chunks) with
  loose faces beside them; nets, areas and corrected fluxes;
* the chain of one time step: the O-grid's fringe velocities interpolated from the background (GPU: the fused
  call; oracle: its own interpolation), then the flux through the O-grid's interface shell and its correction;
* a face id that leaves the grid is reported by ovs_sync.
Tolerances: fluxes |U - U_ref| <= tol * (|u|max |S| of the face), tol = 1e-12 (FP64) / 1e-5 (FP32: the face areas
are formed in FP32 from the coordinates' FP32 pairs); nets to tol of the sum of |U|, areas to tol relative;
corrected net flux zero to the same.
"""
import numpy as np
import pytest

import gen
import oracle
from harness import GpuScene, OracleScene
from paper_1910_09315_gb300 import ovs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch


def run_flux(scene, gid, faces, signs, starts, vel, correct):
    t = scene.torch
    dev = scene.ctx.device
    fd = t.as_tensor(faces).to(dev)
    sd = t.as_tensor(signs).to(dev) if signs is not None else None
    vd = tuple(t.as_tensor(np.ascontiguousarray(vel[:, c])).to(dev) for c in range(3))
    flux, net = scene.ctx.interface_flux(gid, fd, vd, signs=sd, surf_start=starts, correct=correct)
    scene.ctx.sync()
    return flux.cpu().numpy().astype(np.float64), (net.cpu().numpy() if net is not None else None)


def compare(g, faces, signs, starts, vel, got, nets, got_c, tol):
    xyz = g.xyz()
    U = oracle.face_fluxes(g.dims, g.periodic, xyz, vel.astype(np.float64), faces)
    S = np.array([np.linalg.norm(oracle.face_area_vector(xyz, oracle.face_nodes(g.dims, g.periodic, f))) for f in faces])
    umax = np.abs(vel).max()
    assert np.all(np.abs(got - U) <= tol * umax * S + 1e-300), np.abs(got - U).max()
    Uc, nref, aref = oracle.mass_correct(g.dims, g.periodic, xyz, U, faces, signs, starts)
    for s in range(len(starts) - 1):
        sl = slice(starts[s], starts[s + 1])
        scale = np.sum(np.abs(U[sl]))
        assert abs(nets[2 * s] - nref[s]) <= tol * scale
        assert abs(nets[2 * s + 1] - aref[s]) <= tol * aref[s]  # areas: FP64 for FP64 velocities, else FP32
        assert np.all(np.abs(got_c[sl] - Uc[sl]) <= tol * umax * S[sl] + tol * scale * S[sl] / aref[s])
        assert abs(np.sum(signs[sl] * got_c[sl])) <= 4 * tol * scale
    loose = np.ones(len(faces), bool)
    loose[starts[0]:starts[-1]] = False
    assert np.array_equal(got_c[loose], got[loose])  # faces outside every surface keep their flux


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_face_fluxes_and_correction_match_oracle(torch_cuda, dtype):
    sc = gen.config(1)
    scene = GpuScene(sc, max_points=16)
    rng = np.random.default_rng(12)
    tol = 1e-12 if dtype == np.float64 else 1e-5
    for gid in (0, 1):  # the stretched background, then the O-grid (periodic azimuth)
        g = sc.grids[gid]
        n = g.dims
        if gid == 0:
            boxes = [((3, 5, 7), (40, 33, 29)), ((60, 70, 80), (101, 96, 127))]
        else:
            boxes = [((0, 0, n[2] - 2), (n[0], n[1] - 1, n[2] - 1)), ((5, 3, 10), (40, 30, 33))]
        parts = [gen.index_box_surface(n, g.periodic, lo, hi) for lo, hi in boxes]
        ijk = [rng.integers(0, n[m] - 1, 500) for m in range(3)]  # loose interior faces
        extra = (3 * (ijk[0] + n[0] * (ijk[1] + n[1] * ijk[2])) + rng.integers(0, 3, 500)).astype(np.int64)
        faces = np.concatenate([parts[0][0], parts[1][0], extra])
        signs = np.concatenate([parts[0][1], parts[1][1], np.ones(len(extra), np.int8)]).astype(np.int8)
        # the second surface is empty (no faces): its net and area are 0 and nothing is corrected
        starts = [0, len(parts[0][0]), len(parts[0][0]), len(parts[0][0]) + len(parts[1][0])]
        xyz = g.xyz()
        vel = (np.sin(3 * xyz) + rng.uniform(-0.5, 0.5, xyz.shape)).astype(dtype)
        got, nets = run_flux(scene, gid, faces, signs, starts, vel, correct=False)
        got_c, nets_c = run_flux(scene, gid, faces, signs, starts, vel, correct=True)
        assert np.array_equal(nets, nets_c)  # the nets are those before the correction, and reproducible
        compare(g, faces, signs, starts, vel, got, nets, got_c, tol)


def test_interface_flux_of_interpolated_fringe_velocities(torch_cuda):
    """One step of the moving ellipsoid: the O-grid's outer two radial layers take their velocities from the
    background (the fused call on the GPU, the oracle's interpolation on the CPU); the flux through the closed
    shell between those layers (wrapping around the azimuth, closed by the two polar rings) is reconstructed and
    corrected to zero net flux."""
    sc = gen.config(1)
    m = sc.motion(3)
    fsets = sc.fringe_sets(3, m)
    scene = GpuScene(sc, max_points=sum(len(s.node_ids) for s in fsets) + 16)
    scene.set_motion(m)
    sets = scene.upload_sets(fsets)
    d, out = scene.ctx.assemble_interpolate(sets, scene.fields)
    scene.ctx.sync()
    og = sc.grids[1]
    n = og.dims
    t = torch_cuda
    gvel = [t.zeros(og.n_nodes, dtype=t.float32, device=scene.ctx.device) for _ in range(3)]
    ref, frames = OracleScene(sc).step(m, fsets)
    rvel = np.zeros((og.n_nodes, 3))
    b = 0
    for s, (od, oq) in zip(fsets, ref):
        k = len(s.node_ids)
        if s.receiver == 1:
            idx = t.as_tensor(s.node_ids.astype(np.int64)).to(scene.ctx.device)
            for c in range(3):
                gvel[c].index_copy_(0, idx, out[c][b:b + k])
            rvel[s.node_ids] = oq[:3].T
        b += k
    faces, signs = gen.index_box_surface(n, og.periodic, (0, 0, n[2] - 2), (n[0], n[1] - 1, n[2] - 1))
    fd = t.as_tensor(faces).to(scene.ctx.device)
    sd = t.as_tensor(signs).to(scene.ctx.device)
    flux, net = scene.ctx.interface_flux(1, fd, tuple(gvel), signs=sd, surf_start=[0, len(faces)], correct=True)
    scene.ctx.sync()
    xyz = og.xyz()
    U = oracle.face_fluxes(n, og.periodic, xyz, rvel, faces)
    Uc, nref, aref = oracle.mass_correct(n, og.periodic, xyz, U, faces, signs, [0, len(faces)])
    S = np.array([np.linalg.norm(oracle.face_area_vector(xyz, oracle.face_nodes(n, og.periodic, f))) for f in faces])
    scale = np.abs(rvel).max() + 10.0  # velocities plus the frame terms the interpolation tolerance carries
    got = flux.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - Uc) <= 1e-5 * scale * S * 4)
    netg = net.cpu().numpy()
    assert abs(netg[0] - nref[0]) <= 1e-5 * scale * aref[0]
    assert abs(np.sum(signs * got)) <= 1e-5 * np.sum(np.abs(U))


def test_bad_face_is_reported(torch_cuda):
    sc = gen.config(0)
    scene = GpuScene(sc, max_points=16)
    g = sc.grids[0]
    vel = np.zeros((g.n_nodes, 3))
    n = g.dims
    edge = 3 * ((n[0] - 1) + n[0] * 0) + 1  # base at i = n-1, d = 1 spans k and i: leaves the grid along i
    run = lambda: run_flux(scene, 0, np.array([edge], np.int64), None, None, vel, correct=False)
    with pytest.raises(ovs.OvsError) as e:
        run()
    assert e.value.code == ovs.OVS_ERR_DEVICE
    with pytest.raises(ovs.OvsError):
        scene.ctx.interface_flux(0, scene.torch.zeros(1, dtype=scene.torch.int64, device=scene.ctx.device),
                                 tuple(scene.torch.zeros(4, device=scene.ctx.device) for _ in range(3)),
                                 correct=True)  # a correction needs a surface


def test_a_surface_of_thousands_of_chunks(torch_cuda):
    """A closed surface listed 80 times over (4.5 M faces: more than 4096 chunks of 1024 faces, so the chunk length
    grows) sums to 80 times the net and area of one copy, every copy keeps the single copy's face fluxes bit for
    bit, and the correction (net over area, the same ratio) matches the oracle's on one copy."""
    sc = gen.config(1)
    scene = GpuScene(sc, max_points=16)
    g = sc.grids[0]
    faces1, signs1 = gen.index_box_surface(g.dims, g.periodic, (3, 5, 7), (100, 96, 110))
    R = 80
    faces = np.tile(faces1, R)
    signs = np.tile(signs1, R).astype(np.int8)
    xyz = g.xyz()
    vel = np.sin(3 * xyz) + 0.2
    got, nets = run_flux(scene, 0, faces, signs, [0, len(faces)], vel, correct=False)
    got_c, nets_c = run_flux(scene, 0, faces, signs, [0, len(faces)], vel, correct=True)
    m = len(faces1)
    one = got[:m]
    assert all(np.array_equal(got[r * m:(r + 1) * m], one) for r in range(R))
    U = oracle.face_fluxes(g.dims, g.periodic, xyz, vel, faces1)
    Uc, nref, aref = oracle.mass_correct(g.dims, g.periodic, xyz, U, faces1, signs1, [0, m])
    scale = np.sum(np.abs(U))
    assert abs(nets[0] - R * nref[0]) <= 1e-9 * R * scale
    assert abs(nets[1] - R * aref[0]) <= 1e-9 * R * aref[0]
    assert np.array_equal(nets, nets_c)
    S = np.array([np.linalg.norm(oracle.face_area_vector(xyz, oracle.face_nodes(g.dims, g.periodic, f))) for f in faces1])
    tol = 1e-9 * (np.abs(vel).max() * S + scale * S / aref[0])
    assert all(np.all(np.abs(got_c[r * m:(r + 1) * m] - Uc) <= tol) for r in (0, R // 2, R - 1))
