"""The synthetic inputs are valid overset grids: every cell has a positive corner Jacobian at all 8 corners
(no folded or degenerate cells), the fringe sets are in range, and the inputs are reproducible."""
import numpy as np
import pytest

import gen


def corner_jacobians(g):
    ni, nj, nk = g.dims
    X = np.stack([g.x, g.y, g.z], axis=1).reshape(ni, nj, nk, 3, order="F")
    if g.periodic[0]:
        X = np.concatenate([X, X[:1]], axis=0)
    if g.periodic[1]:
        X = np.concatenate([X, X[:, :1]], axis=1)
    if g.periodic[2]:
        X = np.concatenate([X, X[:, :, :1]], axis=2)
    dets = []
    for di in (0, 1):
        for dj in (0, 1):
            for dk in (0, 1):
                sl = lambda o, n: slice(o, n - 1 + o)
                c = X[sl(di, X.shape[0]), sl(dj, X.shape[1]), sl(dk, X.shape[2])]
                e = []
                for ax, d in ((0, di), (1, dj), (2, dk)):
                    o = [di, dj, dk]
                    o[ax] = 1 - d
                    other = X[sl(o[0], X.shape[0]), sl(o[1], X.shape[1]), sl(o[2], X.shape[2])]
                    e.append((other - c) * (1 if d == 0 else -1))
                dets.append(np.einsum("...i,...i->...", e[0], np.cross(e[1], e[2])))
    return np.stack(dets)


@pytest.mark.parametrize("cfg", [0, 1])
def test_grids_valid(cfg):
    sc = gen.config(cfg)
    for g in sc.grids:
        d = corner_jacobians(g)
        sgn = np.sign(d.mean())
        assert sgn != 0
        assert np.all(d * sgn > 0), g.name


@pytest.mark.parametrize("cfg", [0, 1])
def test_sets_in_range_and_reproducible(cfg):
    a = gen.config(cfg)
    b = gen.config(cfg)
    for step in (0, a.nsteps - 1):
        sa, sb = a.fringe_sets(step), b.fringe_sets(step)
        for x, y in zip(sa, sb):
            assert np.array_equal(x.node_ids, y.node_ids)
            assert x.node_ids.dtype == np.int32
            assert x.node_ids.min() >= 0 and x.node_ids.max() < a.grids[x.receiver].n_nodes
            assert np.all(np.diff(x.node_ids) > 0)
    ma, mb = a.motion(a.nsteps - 1), b.motion(a.nsteps - 1)
    for x, y in zip(ma, mb):
        assert np.array_equal(x.R, y.R) and np.array_equal(x.c, y.c)
        assert np.abs(x.R.T @ x.R - np.eye(3)).max() < 1e-14


def test_cfg1_motion_matches_stated_rates():
    sc = gen.config(1)
    m0, m1 = sc.motion(0)[1], sc.motion(1)[1]
    assert np.linalg.norm(m0.omega) == pytest.approx(2 * np.pi)
    assert np.linalg.norm(m0.V) == pytest.approx(0.3)
    # one step of dt turns the frame by |omega| dt about omega and moves it by V dt
    dR = m1.R @ m0.R.T
    ang = np.arccos((np.trace(dR) - 1) / 2)
    assert ang == pytest.approx(2 * np.pi * 1e-3, rel=1e-9)
    assert np.allclose(m1.c - m0.c, m0.V * 1e-3, atol=1e-15)
