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


@pytest.mark.parametrize("dims", [(48, 32, 32), (160, 96, 96)])
def test_fish_grids_valid(dims):
    g = gen.fish_ogrid("fish", *dims, phase=1.3)
    d = corner_jacobians(g)
    sgn = np.sign(d.mean())
    assert np.all(d * sgn > 0)


def test_fish_layer_test_matches_grid():
    """The analytic layer test agrees with the grid's own k-layers: nodes inside layer nk-3 for k < nk-3,
    outside for k > nk-3; outside the body for k >= 1; the midline itself is inside the body."""
    phase = 0.7
    g = gen.fish_ogrid("fish", 64, 40, 40, phase)
    ni, nj, nk = g.dims
    p = g.xyz()
    k = np.arange(g.n_nodes) // (ni * nj)
    f = g.meta["t"][-3]
    inside = gen.inside_fish_layer(p, phase, f)
    assert np.all(inside[k < nk - 3]) and not np.any(inside[k > nk - 3])
    body = gen.inside_fish_layer(p, phase, 0.0)
    assert not np.any(body[k >= 1])
    s = np.linspace(0.05, 0.95, 50)
    mid = np.stack([s - 0.5, gen.fish_midline(s, phase), np.zeros_like(s)], axis=1)
    assert np.all(gen.inside_fish_layer(mid, phase, 0.0))


def test_fish_envelope_reading():
    """a(s) = 0.02 - 0.08 s + 0.16 s^2 reaches the stated tail excursion 0.1 L at s = 1."""
    assert gen.fish_envelope(np.array([1.0]))[0] == pytest.approx(0.10)
    assert gen.fish_envelope(np.array([0.0]))[0] == pytest.approx(0.02)


@pytest.fixture(scope="module")
def school():
    return gen.config(3)


def test_school_sets(school):
    sc = school
    nfish = len(sc.grids) - 1
    for step in (0, sc.nsteps - 1):
        m = sc.motion(step)
        sets = sc.fringe_sets(step, m)
        assert len(sets) <= 64
        kinds = {s.kind for s in sets}
        assert {"body->bg", "body->body", "bg->body"} <= kinds
        seen = {}
        for s in sets:
            g = sc.grids[s.receiver]
            assert s.node_ids.dtype == np.int32 and len(s.node_ids) > 0
            assert s.node_ids.min() >= 0 and s.node_ids.max() < g.n_nodes
            assert np.all(np.diff(s.node_ids) > 0)
            assert 1 <= len(s.donors) <= 8 and s.receiver not in s.donors
            if s.receiver > 0:
                assert s.donors[-1] == 0  # body fringe falls back to the background
            else:
                assert all(1 <= d <= nfish for d in s.donors) and s.donors == sorted(s.donors)
            prev = seen.setdefault(s.receiver, set())
            ids = set(s.node_ids.tolist())
            assert not (prev & ids)  # a receiver node is in one set only
            prev |= ids
        # background receivers lie inside the hull of their first donor and outside every body
        bgset = [s for s in sets if s.receiver == 0]
        bg = sc.grids[0]
        phase = sc.meta["phase"]
        for s in bgset[:4]:
            pts = bg.xyz()[s.node_ids[:2000]]
            q = s.donors[0]
            b = gen.to_body(m[q], pts)
            assert np.all(gen.inside_fish_layer(b, phase, sc.grids[q].meta["t"][-3]))
            for r in range(1, nfish + 1):
                assert not np.any(gen.inside_fish_layer(gen.to_body(m[r], pts), phase, 0.0))


def test_school_motion(school):
    sc = school
    dt = sc.dt
    m0, m1 = sc.motion(10), sc.motion(11)
    for a, b in zip(m0[1:], m1[1:]):
        assert np.allclose(b.c - a.c, a.V * dt, atol=1e-15)
        dR = b.R @ a.R.T
        ang = np.arctan2(dR[1, 0], dR[0, 0])
        assert ang == pytest.approx(0.5 * (a.omega[2] + b.omega[2]) * dt, rel=1e-3, abs=1e-9)
        assert np.abs(a.R.T @ a.R - np.eye(3)).max() < 1e-14


def naca12_half_width(s):
    """NACA four-digit half-thickness at 12 % of the chord (closed trailing edge), written out from its definition."""
    return 5 * 0.12 * (0.2969 * np.sqrt(s) - 0.1260 * s - 0.3516 * s ** 2 + 0.2843 * s ** 3 - 0.1036 * s ** 4)


@pytest.mark.parametrize("which", ["ellipsoid", "fish"])
def test_body_surface_closed_oriented_and_of_the_body_volume(which):
    """The hole-cutting surfaces: every directed edge used once and its reverse once (closed, consistently
    oriented), no zero-area triangle, and the enclosed volume (divergence theorem) just below the body's own --
    the vertices lie on the body, so the facets are chords: the ellipsoid 4/3 pi abc, the fish the integral of
    its elliptic cross-sections pi w (1.6 w) (the midline shear keeps volume)."""
    from scipy.integrate import quad

    if which == "ellipsoid":
        g = gen.ellipsoid_ogrid(48, 32, 8, (0.2, 0.1, 0.1), 0.4, beta_r=2.0)
        want = 4.0 / 3.0 * np.pi * 0.2 * 0.1 * 0.1
    else:
        g = gen.fish_ogrid("fish", 64, 48, 8, phase=1.1)
        want = quad(lambda s: np.pi * naca12_half_width(s) * 1.6 * naca12_half_width(s), 0.0, 1.0)[0]
    V, T = gen.body_surface(g)
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]]).tolist()
    directed = set(map(tuple, e))
    assert len(directed) == len(e) and all((b, a) in directed for a, b in directed)
    P = V[T]
    assert np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1).min() > 0
    vol = abs(np.einsum("ij,ij->i", P[:, 0], np.cross(P[:, 1], P[:, 2])).sum() / 6.0)
    assert 0.985 * want < vol <= want * (1 + 1e-9), (vol, want)
