"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test ties one part of the oracle to something other than itself:
closed forms on Cartesian cells, the paper's face-distance coefficients on
affine cells (Sec. 2.2.6), exact reproduction of linear fields, the
partition of unity of the trilinear weights, rigid-frame identities of
Sec. 2.1 / Sec. 2.3.1, brute force on tiny grids, and finite differences for
the guess network's gradients.
"""
import math

import numpy as np
import pytest

import gen
import oracle
from gen import axis_angle, euler_zyx


def cart_grid(n, lo, hi):
    axes = [lo[d] + (hi[d] - lo[d]) * np.arange(n[d]) / (n[d] - 1) for d in range(3)]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    f = lambda a: a.ravel(order="F")
    return oracle.OracleGrid(n, (False, False, False), f(X), f(Y), f(Z))


def lerp_hex(X, xi):
    """Trilinear map by nested linear interpolation along i, then j, then k (independent of the product form)."""
    X = np.asarray(X).reshape(2, 2, 2, 3, order="F")  # [di, dj, dk, c], corner a = di + 2dj + 4dk
    a = X[0] * (1 - xi[0]) + X[1] * xi[0]  # [dj, dk, c]
    b = a[0] * (1 - xi[1]) + a[1] * xi[1]  # [dk, c]
    return b[0] * (1 - xi[2]) + b[1] * xi[2]


def distorted_hex(rng, amp=0.2, scale=1.0, origin=None):
    X = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float)
    X = X + amp * rng.uniform(-1, 1, size=(8, 3))
    X = X * scale
    if origin is not None:
        X = X + origin
    return X


# ----------------------------------------------------------------------------- weights
def test_shape_functions_kronecker_and_unity():
    rng = np.random.default_rng(1)
    for a in range(8):
        corner = np.array([a & 1, (a >> 1) & 1, (a >> 2) & 1], float)
        N = oracle.shape(corner)
        assert np.array_equal(N, np.eye(8)[a])
    for _ in range(100):
        xi = rng.uniform(-0.5, 1.5, 3)
        N = oracle.shape(xi)
        assert abs(N.sum() - 1.0) < 1e-15
    # the sign-corrected form of the paper's trilinear formula: node (i,j,k) weighs (1-x)(1-y)(1-z)
    N = oracle.shape(np.array([0.25, 0.5, 0.75]))
    assert N[0] == pytest.approx(0.75 * 0.5 * 0.25, abs=1e-16)
    assert N[7] == pytest.approx(0.25 * 0.5 * 0.75, abs=1e-16)
    assert N[1] == pytest.approx(0.25 * 0.5 * 0.25, abs=1e-16)


# ----------------------------------------------------------------------------- Newton
def test_newton_recovers_xi_on_distorted_hexes():
    rng = np.random.default_rng(2)
    for t in range(300):
        X = distorted_hex(rng, amp=0.2, scale=10 ** rng.uniform(-3, 0), origin=rng.uniform(-5, 5, 3))
        xi_true = rng.uniform(0, 1, 3)
        p = lerp_hex(X, xi_true)
        ok, xi, it = oracle.newton_hex(X, p)
        assert ok and it <= 10
        assert np.max(np.abs(xi - xi_true)) < 1e-12


def test_affine_cells_match_paper_face_distance_coefficients():
    """On a parallelepiped the paper's a^1 = d^1/(d^1+d^2) (distances to the two i-faces, Sec. 2.2.6) is the
    exact local coordinate; the same for j and k."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        E = rng.uniform(-1, 1, (3, 3)) + 2 * np.eye(3)
        X0 = rng.uniform(-3, 3, 3)
        X = np.array([X0 + (a & 1) * E[0] + ((a >> 1) & 1) * E[1] + ((a >> 2) & 1) * E[2] for a in range(8)])
        p = X0 + rng.uniform(-0.3, 1.3, 3) @ E
        ok, xi, _ = oracle.newton_hex(X, p)
        assert ok
        for m in range(3):
            u, v = E[(m + 1) % 3], E[(m + 2) % 3]
            n = np.cross(u, v)
            n = n / np.linalg.norm(n)
            if np.dot(n, E[m]) < 0:
                n = -n  # inward normal of the face at offset 0
            d1 = np.dot(p - X0, n)  # signed distance to the face through X0
            d2 = np.dot(X0 + E[m] - p, n)  # signed distance to the opposite face
            assert xi[m] == pytest.approx(d1 / (d1 + d2), abs=1e-13)


def test_linear_fields_reproduced_exactly():
    rng = np.random.default_rng(4)
    for _ in range(200):
        X = distorted_hex(rng, amp=0.25, scale=0.01, origin=rng.uniform(0, 4, 3))
        p = lerp_hex(X, rng.uniform(0, 1, 3))
        ok, xi, _ = oracle.newton_hex(X, p)
        assert ok
        N = oracle.shape(xi)
        a, b = rng.uniform(-1, 1, 3), rng.uniform(-1, 1)
        q = X @ a + b
        assert np.dot(N, q) == pytest.approx(np.dot(a, p) + b, abs=1e-13 * (1 + abs(np.dot(a, p) + b)))
        assert np.allclose(N @ X, p, rtol=0, atol=1e-15 * 4)


def test_newton_fails_on_flat_hex():
    X = np.array([[a & 1, (a >> 1) & 1, 0.0] for a in range(8)], dtype=float)  # zero thickness
    ok, xi, _ = oracle.newton_hex(X, np.array([0.5, 0.5, 0.0]))
    assert not ok


# ----------------------------------------------------------------------------- donor selection
def closed_form_cell(t, n):
    """Lowest cell whose window [-1e-10, 1+1e-10] holds the scaled coordinate t on a uniform axis of n nodes."""
    i = max(0, math.ceil(t - 1 - 1e-10))
    return min(i, n - 2)


def test_uniform_cartesian_closed_form_generic_points():
    n, lo, hi = (9, 7, 6), (0.1, -0.3, 2.0), (1.3, 0.9, 2.5)
    g = cart_grid(n, lo, hi)
    h = [(hi[d] - lo[d]) / (n[d] - 1) for d in range(3)]
    rng = np.random.default_rng(5)
    pts = np.stack([rng.uniform(lo[d], hi[d], 2000) for d in range(3)], axis=1)
    cell, xi, nodes, w = g.search(pts)
    for q in range(len(pts)):
        t = [(pts[q, d] - lo[d]) / h[d] for d in range(3)]
        ijk = [min(int(math.floor(t[d])), n[d] - 2) for d in range(3)]
        expect = ijk[0] + (n[0] - 1) * (ijk[1] + (n[1] - 1) * ijk[2])
        assert cell[q] == expect
        for d in range(3):
            assert xi[q, d] == pytest.approx(t[d] - ijk[d], abs=1e-12)
        assert abs(w[q].sum() - 1) < 1e-14


def test_uniform_cartesian_ties_on_nodes_and_faces():
    n, lo, hi = (6, 5, 7), (0.0, 0.0, 0.0), (1.0, 2.0, 3.0)
    g = cart_grid(n, lo, hi)
    h = [(hi[d] - lo[d]) / (n[d] - 1) for d in range(3)]
    rng = np.random.default_rng(6)
    pts, ts = [], []
    for _ in range(400):
        t = []
        for d in range(3):
            kind = rng.integers(3)
            if kind == 0:
                t.append(float(rng.integers(0, n[d])))  # on a node plane
            else:
                t.append(rng.uniform(0, n[d] - 1))
        ts.append(t)
        pts.append([lo[d] + t[d] * h[d] for d in range(3)])
    pts = np.array(pts)
    cell, xi, _, _ = g.search(pts)
    for q, t in enumerate(ts):
        tt = [(pts[q, d] - lo[d]) / h[d] for d in range(3)]
        ijk = [closed_form_cell(tt[d], n[d]) for d in range(3)]
        expect = ijk[0] + (n[0] - 1) * (ijk[1] + (n[1] - 1) * ijk[2])
        assert cell[q] == expect, (t, cell[q], expect)


def test_interior_node_goes_to_lowest_of_eight_cells():
    n = (5, 5, 5)
    g = cart_grid(n, (0, 0, 0), (1, 1, 1))
    p = np.array([[0.5, 0.25, 0.75]])  # node (2,1,3)
    cell, xi, _, _ = g.search(p)
    assert cell[0] == 1 + 4 * (0 + 4 * 2)  # cell (1,0,2): the one with the lowest linear id
    assert np.allclose(xi[0], [1, 1, 1], atol=1e-12)


def test_outside_and_nonfinite_points():
    g = cart_grid((4, 4, 4), (0, 0, 0), (1, 1, 1))
    cell, xi, _, _ = g.search(np.array([[1.5, 0.5, 0.5], [-1e-6, 0.5, 0.5], [np.nan, 0.5, 0.5], [1 + 1e-12, 0.5, 0.5]]))
    assert list(cell[:3]) == [-1, -1, -2]
    assert cell[3] >= 0  # within the 1e-10 window of the boundary cell


def random_curvilinear(n, amp, rng, periodic_i=False):
    """A smooth invertible curvilinear grid: unit-box (or annulus sector when periodic in i) plus a sine warp."""
    I, J, K = np.meshgrid(*[np.arange(m, dtype=float) for m in n], indexing="ij")
    if periodic_i:
        th = 2 * np.pi * I / n[0]
        r = 1.0 + J / (n[1] - 1)
        x, y, z = r * np.cos(th), r * np.sin(th), K / (n[2] - 1)
    else:
        x, y, z = I / (n[0] - 1), J / (n[1] - 1), K / (n[2] - 1)
    h = 1.0 / max(n)
    ph = rng.uniform(0, 2 * np.pi, 3)
    x = x + amp * h * np.sin(2 * np.pi * y + ph[0]) * np.cos(2 * np.pi * z)
    y = y + amp * h * np.sin(2 * np.pi * z + ph[1]) * np.cos(2 * np.pi * x)
    z = z + amp * h * np.sin(2 * np.pi * x + ph[2])
    f = lambda a: a.ravel(order="F")
    return oracle.OracleGrid(n, (periodic_i, False, False), f(x), f(y), f(z), bins=(3, 3, 3))


@pytest.mark.parametrize("periodic", [False, True])
def test_bins_equal_brute_force_on_tiny_grids(periodic):
    rng = np.random.default_rng(7 + periodic)
    n = (5, 5, 5) if periodic else (8, 8, 8)
    g = random_curvilinear(n, 0.8, rng, periodic_i=periodic)
    xyz = np.stack([g.x, g.y, g.z], axis=1)
    lo, hi = xyz.min(0), xyz.max(0)
    pts = [rng.uniform(lo - 0.05, hi + 0.05, size=(1500, 3)), xyz[rng.integers(0, len(xyz), 200)]]
    # points on cell faces: midpoints of node pairs along each axis
    a = rng.integers(0, len(xyz), 200)
    pts.append(0.5 * (xyz[a] + xyz[np.minimum(a + 1, len(xyz) - 1)]))
    pts = np.concatenate(pts)
    c1, x1, _, _ = g.search(pts, brute=False)
    c2, x2, _, _ = g.search(pts, brute=True)
    assert np.array_equal(c1, c2)
    found = c1 >= 0
    assert found.sum() > 500
    assert np.allclose(x1[found], x2[found], atol=0, rtol=0)


def test_periodic_seam_cell():
    rng = np.random.default_rng(9)
    n = (6, 4, 3)
    g = random_curvilinear(n, 0.0, rng, periodic_i=True)
    # the seam cell i = n0-1 joins node i = 5 to node i = 0
    nodes = g.cell_nodes(5)
    assert nodes[0] == 5 and nodes[1] == 0
    xyz = np.stack([g.x, g.y, g.z], axis=1)
    X = xyz[nodes]
    p = lerp_hex(X, np.array([0.4, 0.3, 0.6]))
    cell, xi, _, _ = g.search(p[None])
    assert cell[0] == 5
    assert np.allclose(xi[0], [0.4, 0.3, 0.6], atol=1e-12)


# ----------------------------------------------------------------------------- frames
def test_frame_round_trip_and_closed_form():
    rng = np.random.default_rng(10)
    R = euler_zyx(*rng.uniform(0, np.pi, 3))
    assert np.abs(R.T @ R - np.eye(3)).max() < 1e-15
    f = oracle.Frame(R, rng.uniform(-1, 1, 3), np.zeros(3), np.zeros(3))
    x = rng.uniform(-1, 1, (100, 3))
    assert np.abs(oracle.to_frame(f, oracle.to_inertial(f, x)) - x).max() < 1e-15
    # a quarter turn about z carries body x-axis onto inertial y-axis
    f = oracle.Frame(axis_angle(np.array([0, 0, 1.0]), np.pi / 2), np.array([1.0, 2.0, 3.0]), np.zeros(3), np.zeros(3))
    assert np.allclose(oracle.to_inertial(f, np.array([[1.0, 0, 0]])), [[1.0, 3.0, 3.0]], atol=1e-15)


def _rigid_case(rng):
    """Donor body grid (distorted hexes) carrying the relative velocity of the inertial rigid field
    u(x) = V0 + W0 x x, i.e. u_rel = R^T (u(x_in) - V - omega x (x_in - c)) at each node."""
    V0, W0 = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    g = random_curvilinear((6, 6, 6), 0.5, rng)
    fd = oracle.Frame(euler_zyx(*rng.uniform(0, np.pi, 3)), rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3),
                      rng.uniform(-1, 1, 3))
    X = np.stack([g.x, g.y, g.z], axis=1)
    x_in = oracle.to_inertial(fd, X)
    u_in = V0 + np.cross(W0, x_in)
    u_rel = (u_in - fd.V - np.cross(fd.omega, x_in - fd.c)) @ fd.R
    fields = {"u": u_rel[:, 0], "v": u_rel[:, 1], "w": u_rel[:, 2], "p": np.zeros(len(X))}
    return V0, W0, g, fd, fields


def test_rigid_body_velocity_reproduced_in_inertial_receiver():
    rng = np.random.default_rng(11)
    V0, W0, g, fd, fields = _rigid_case(rng)
    # receiver: an inertial (background) grid whose nodes lie inside the body grid
    X = np.stack([g.x, g.y, g.z], axis=1)
    inner = oracle.to_inertial(fd, X[[7 + 6 * 7 + 36 * k for k in range(1, 4)]] * 0.999 + 0.001 * X.mean(0))
    fr = oracle.Frame(np.eye(3), np.zeros(3), np.zeros(3), np.zeros(3))
    d = oracle.assemble([None, g], [fr, fd], inner, 0, np.arange(len(inner)), [1])
    assert np.all(d.status == 0)
    q = oracle.interpolate(d, [None, fields], [fr, fd], 0, mode="relative")
    expect = V0 + np.cross(W0, d.x_in)
    assert np.abs(q[:3].T - expect).max() < 1e-13


def test_rigid_body_velocity_between_moving_frames():
    rng = np.random.default_rng(12)
    V0, W0, g, fd, fields = _rigid_case(rng)
    fr = oracle.Frame(euler_zyx(*rng.uniform(0, np.pi, 3)), rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3),
                      rng.uniform(-1, 1, 3))
    X = np.stack([g.x, g.y, g.z], axis=1)
    pts_in = oracle.to_inertial(fd, 0.5 * (X[8] + X[120]))[None]
    rec = oracle.to_frame(fr, pts_in)
    d = oracle.assemble([None, g], [fr, fd], rec, 0, np.arange(1), [1])
    assert d.status[0] == 0
    q = oracle.interpolate(d, [None, fields], [fr, fd], 0, mode="relative")
    u_in = V0 + np.cross(W0, pts_in[0])
    expect = fr.R.T @ (u_in - fr.V - np.cross(fr.omega, pts_in[0] - fr.c))
    assert np.abs(q[:3, 0] - expect).max() < 1e-13


def test_absolute_mode_is_pure_rotation():
    """Sec. 2.3.1: u^m = Q^m (Q^n)^-1 u^n with Q = R^T; a quarter turn of the donor about z maps its body
    x-velocity to the inertial (receiver) y-velocity, independent of V and omega."""
    n = (3, 3, 3)
    g = cart_grid(n, (0, 0, 0), (1, 1, 1))
    fd = oracle.Frame(axis_angle(np.array([0, 0, 1.0]), np.pi / 2), np.zeros(3), np.array([5.0, 6, 7]),
                      np.array([1.0, 2, 3]))
    fr = oracle.Frame(np.eye(3), np.zeros(3), np.zeros(3), np.zeros(3))
    fields = {"u": np.ones(27), "v": np.zeros(27), "w": np.zeros(27), "p": np.full(27, 2.5)}
    pts = oracle.to_inertial(fd, np.array([[0.3, 0.4, 0.5]]))
    d = oracle.assemble([None, g], [fr, fd], pts, 0, np.arange(1), [1])
    q = oracle.interpolate(d, [None, fields], [fr, fd], 0, mode="absolute")
    assert np.allclose(q[:, 0], [0, 1, 0, 2.5], atol=1e-15)


def test_priority_list_falls_through_to_next_grid():
    g1 = cart_grid((4, 4, 4), (0, 0, 0), (1, 1, 1))
    g2 = cart_grid((4, 4, 4), (0.5, 0, 0), (2, 1, 1))
    I = oracle.Frame(np.eye(3), np.zeros(3), np.zeros(3), np.zeros(3))
    pts = np.array([[0.7, 0.5, 0.5], [1.7, 0.5, 0.5], [3.0, 0.5, 0.5], [np.inf, 0, 0]])
    d = oracle.assemble([None, g1, g2], [I, I, I], pts, 0, np.arange(4), [1, 2])
    assert list(d.grid) == [1, 2, -1, -1]
    assert list(d.status) == [0, 0, 1, 2]


# ----------------------------------------------------------------------------- guess network
def _mlp(rng, H):
    return {"W1": rng.normal(0, 0.8, (H, 3)), "b1": rng.normal(0, 0.1, H), "W2": rng.normal(0, 0.3, (H, H)),
            "b2": rng.normal(0, 0.1, H), "W3": rng.normal(0, 0.3, (3, H)), "b3": rng.normal(0, 0.1, 3)}


@pytest.mark.parametrize("H", [8, 64])
def test_mlp_gradients_match_finite_differences(H):
    rng = np.random.default_rng(13)
    P = _mlp(rng, H)
    x = rng.uniform(-1, 1, (16, 3))
    t = rng.uniform(0, 1, (16, 3))
    L, g = oracle.mlp_loss_grads(P, x, t)
    h = 1e-6
    for k in P:
        flatp = P[k].reshape(-1)
        idx = rng.choice(flatp.size, size=min(flatp.size, 12), replace=False)
        for i in idx:
            old = flatp[i]
            flatp[i] = old + h
            Lp, _ = oracle.mlp_loss_grads(P, x, t)
            flatp[i] = old - h
            Lm, _ = oracle.mlp_loss_grads(P, x, t)
            flatp[i] = old
            fd = (Lp - Lm) / (2 * h)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd), abs(an)), (k, i, fd, an)


def test_silu_closed_form():
    z = np.array([-3.0, 0.0, 2.0])
    assert np.allclose(oracle.silu(z), z / (1 + np.exp(-z)))
    assert oracle.silu(np.array([0.0]))[0] == 0.0
    assert oracle.dsilu(np.array([0.0]))[0] == pytest.approx(0.5)


def test_mlp_forward_hand_worked_h2_network():
    """A 3-2-2-3 network whose output is worked out by hand.  sigma(ln 3) = 1 / (1 + 1/3) = 3/4 and
    sigma(-ln 3) = 1/4, so silu(ln 3) = (3/4) ln 3, silu(-ln 3) = -(1/4) ln 3 and silu(0) = 0.
    Layer 1 picks x0 and x1 (x2 must not matter): z1 = (ln 3, -ln 3), h1 = ((3/4) ln 3, -(1/4) ln 3).
    Layer 2 (W2[out][in] = [[1, 1], [2, 0]], b2 = ((1/2) ln 3, -(3/2) ln 3)): z2 = (ln 3, 0),
    h2 = ((3/4) ln 3, 0).  Output layer, linear (no SiLU): y = W3 h2 + b3 with W3 = [[1, 0], [0, 1], [2, 3]],
    b3 = (1, 2, 3): y = ((3/4) ln 3 + 1, 2, (3/2) ln 3 + 3).
    A SiLU on the output (y1 = silu(2) != 2), a transposed W2 (z2_0 = (3/4) ln 3), a dropped bias, or x2
    leaking in all change y."""
    L3 = math.log(3.0)
    P = {"W1": np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]), "b1": np.zeros(2),
         "W2": np.array([[1.0, 1.0], [2.0, 0.0]]), "b2": np.array([0.5 * L3, -1.5 * L3]),
         "W3": np.array([[1.0, 0.0], [0.0, 1.0], [2.0, 3.0]]), "b3": np.array([1.0, 2.0, 3.0])}
    x = np.array([[L3, -L3, 5.0], [L3, -L3, -7.0]])
    y, (_, z1, h1, z2, h2) = oracle.mlp_forward(P, x)
    want = np.array([0.75 * L3 + 1.0, 2.0, 1.5 * L3 + 3.0])
    assert np.allclose(y, want[None, :], rtol=0, atol=1e-14)
    assert np.allclose(h1[0], [0.75 * L3, -0.25 * L3], rtol=0, atol=1e-15)
    assert np.allclose(z2[0], [L3, 0.0], rtol=0, atol=1e-15)
    assert np.allclose(h2[0], [0.75 * L3, 0.0], rtol=0, atol=1e-15)


def test_adam_three_steps_against_closed_form_moments():
    """Adam's moments unrolled: m_t = (1 - b1) sum_k b1^(t-k) g_k and v_t = (1 - b2) sum_k b2^(t-k) g_k^2, each
    divided by its bias correction 1 - b^t (Kingma & Ba 2015, Algorithm 1); the step is lr m^_t / (sqrt(v^_t)
    + eps).  Evaluated in exact rationals for a gradient sequence that changes sign and size, so a wrong power
    in either correction (e.g. 1 - b2 in place of 1 - b2^t at t > 1) or a swapped b1 / b2 fails."""
    from fractions import Fraction as Fr

    b1, b2, lr, eps = Fr(9, 10), Fr(999, 1000), 0.05, 1e-8
    gs = [np.array([1.0, 0.25]), np.array([-1.0, 0.5]), np.array([2.0, -3.0])]
    P = {"a": np.array([0.3, -0.7])}
    m = {"a": np.zeros(2)}
    v = {"a": np.zeros(2)}
    want = P["a"].copy()
    for t in range(1, 4):
        oracle.adam_step(P, {"a": gs[t - 1]}, m, v, t, lr=lr, b1=float(b1), b2=float(b2), eps=eps)
        for c in range(2):
            ms = (1 - b1) * sum(b1 ** (t - k) * Fr(gs[k - 1][c]) for k in range(1, t + 1)) / (1 - b1 ** t)
            vs = (1 - b2) * sum(b2 ** (t - k) * Fr(gs[k - 1][c]) ** 2 for k in range(1, t + 1)) / (1 - b2 ** t)
            want[c] -= lr * float(ms) / (math.sqrt(float(vs)) + eps)
        assert np.allclose(P["a"], want, rtol=0, atol=1e-13), (t, P["a"], want)
    # with a constant gradient the corrected moments are g and g^2 at every t: each step is lr sign(g)
    P = {"a": np.array([1.0])}
    m, v = {"a": np.zeros(1)}, {"a": np.zeros(1)}
    for t in range(1, 4):
        oracle.adam_step(P, {"a": np.array([-0.3])}, m, v, t, lr=0.1)
    assert P["a"][0] == pytest.approx(1.3, abs=1e-6)


def test_adam_first_step_is_signed_lr():
    """With bias correction the first Adam step moves each parameter by lr * sign(g) (|g| >> eps)."""
    P = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -4.0, 1e-2])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    oracle.adam_step(P, g, m, v, 1, lr=0.1)
    assert np.allclose(P["a"], [0.9, -1.9, 2.9], atol=1e-6)


# ----------------------------------------------------------------------------- blanked donors (iblank)
def _window(xi):
    return bool(np.all(xi >= -1e-10) and np.all(xi <= 1 + 1e-10))


@pytest.mark.parametrize("periodic", [False, True])
def test_iblank_lowest_usable_cell_by_definition(periodic):
    """With a random iblank, the donor is the lowest-id cell that contains the point (Newton on that cell's own
    corners, ascending ids, written out here cell by cell) and has no blanked corner; bins = brute force."""
    rng = np.random.default_rng(31 + periodic)
    n = (5, 5, 4) if periodic else (6, 6, 5)
    g = random_curvilinear(n, 0.8, rng, periodic_i=periodic)
    iblank = (rng.uniform(size=int(np.prod(n))) > 0.15).astype(np.uint8)
    g.set_iblank(iblank)
    xyz = np.stack([g.x, g.y, g.z], axis=1)
    lo, hi = xyz.min(0), xyz.max(0)
    a = rng.integers(0, len(xyz), 60)
    pts = np.concatenate([rng.uniform(lo, hi, size=(300, 3)), xyz[a],
                          0.5 * (xyz[a] + xyz[np.minimum(a + 1, len(xyz) - 1)])])
    c1, x1, _, _ = g.search(pts, brute=False)
    c2, x2, _, _ = g.search(pts, brute=True)
    assert np.array_equal(c1, c2)
    expect = np.full(len(pts), -1)
    for q, p in enumerate(pts):
        for c in range(g.n_cells):
            nodes = g.cell_nodes(c)
            if not np.all(iblank[nodes]):
                continue
            ok, xi, _ = oracle.newton_hex(xyz[nodes], p)
            if ok and _window(xi):
                expect[q] = c
                break
    assert np.array_equal(c1, expect)
    assert 0 < (c1 >= 0).sum() < len(pts)
    # the blanked cells did change answers: without the mask more points find a donor
    g.set_iblank(None)
    c0, _, _, _ = g.search(pts)
    assert (c0 >= 0).sum() > (c1 >= 0).sum()
    assert np.all((c1 < 0) | (c1 >= c0))  # a usable donor is never below the unmasked lowest id


def test_iblank_all_active_changes_nothing():
    rng = np.random.default_rng(5)
    g = random_curvilinear((7, 6, 5), 0.8, rng)
    xyz = np.stack([g.x, g.y, g.z], axis=1)
    pts = rng.uniform(xyz.min(0), xyz.max(0), size=(500, 3))
    c0, x0, _, _ = g.search(pts)
    g.set_iblank(np.ones(len(xyz), np.uint8))
    c1, x1, _, _ = g.search(pts)
    assert np.array_equal(c0, c1) and np.array_equal(np.isnan(x0), np.isnan(x1))


def test_iblank_falls_through_the_priority_list():
    """A point in a cell of the first grid that touches a blanked node takes its donor from the next grid."""
    g1 = cart_grid((5, 5, 5), (0, 0, 0), (1, 1, 1))
    g2 = cart_grid((4, 4, 4), (0, 0, 0), (1, 1, 1))
    ib = np.ones(125, np.uint8)
    ib[2 + 5 * (2 + 5 * 2)] = 0  # node (2,2,2) at (0.5, 0.5, 0.5): the 8 cells around it cannot donate
    g1.set_iblank(ib)
    I = oracle.Frame(np.eye(3), np.zeros(3), np.zeros(3), np.zeros(3))
    pts = np.array([[0.45, 0.4, 0.6], [0.1, 0.1, 0.1], [0.6, 0.55, 0.3]])
    d = oracle.assemble([None, g1, g2], [I, I, I], pts, 0, np.arange(3), [1, 2])
    assert list(d.grid) == [2, 1, 2] and list(d.status) == [0, 0, 0]
    d1 = oracle.assemble([None, g1], [I, I], pts, 0, np.arange(3), [1])
    assert list(d1.status) == [1, 0, 1]  # with no other grid: orphans


# ----------------------------------------------------------------------------- hole cutting (ray parity)
def _cube_surface():
    V = np.array([[x, y, z] for z in (0.0, 1.0) for y in (0.0, 1.0) for x in (0.0, 1.0)])
    vid = lambda x, y, z: x + 2 * y + 4 * z
    quads = [(vid(0, 0, 0), vid(0, 1, 0), vid(0, 1, 1), vid(0, 0, 1)), (vid(1, 0, 0), vid(1, 1, 0), vid(1, 1, 1), vid(1, 0, 1)),
             (vid(0, 0, 0), vid(1, 0, 0), vid(1, 0, 1), vid(0, 0, 1)), (vid(0, 1, 0), vid(1, 1, 0), vid(1, 1, 1), vid(0, 1, 1)),
             (vid(0, 0, 0), vid(1, 0, 0), vid(1, 1, 0), vid(0, 1, 0)), (vid(0, 0, 1), vid(1, 0, 1), vid(1, 1, 1), vid(0, 1, 1))]
    T = []
    for a, b, c, d in quads:  # each face split along its a-c diagonal
        T += [(a, b, c), (a, c, d)]
    return V, np.array(T, np.int32)


def test_ray_parity_cube_with_ties():
    """Lattice points of spacing 1/4 around the unit cube: strictly inside -> inside, strictly outside -> outside,
    including rays through the faces' shared diagonals, edges and vertices (each crossing counted once)."""
    V, T = _cube_surface()
    g = np.arange(-2, 7) / 4.0
    P = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T
    inside = oracle.surface_inside(V, T, P)
    strict_in = np.all((P > 0) & (P < 1), axis=1)
    strict_out = np.any((P < 0) | (P > 1), axis=1)
    assert np.all(inside[strict_in] == 1) and np.all(inside[strict_out] == 0)
    assert strict_in.sum() == 27 and np.sum(strict_in & (P[:, 1] == P[:, 2])) == 9  # rays along a diagonal


def test_ray_parity_ellipsoid_surface():
    """The triangulated wall of the ellipsoid O-grid: inside iff inside the analytic ellipsoid, away from a band
    around the surface that covers the chords' deviation; invariant under a rigid motion of points and surface."""
    g = gen.ellipsoid_ogrid(48, 32, 8, (0.2, 0.1, 0.1), 0.4, beta_r=2.0)
    V, T = gen.body_surface(g)
    rng = np.random.default_rng(2)
    P = rng.uniform(-0.25, 0.25, size=(20000, 3)) * np.array([1.0, 0.6, 0.6])
    f = (P[:, 0] / 0.2) ** 2 + (P[:, 1] / 0.1) ** 2 + (P[:, 2] / 0.1) ** 2
    clear = np.abs(f - 1) > 0.05
    inside = oracle.surface_inside(V, T, P)
    assert np.array_equal(inside[clear], (f[clear] < 1).astype(np.uint8))
    assert 2000 < inside.sum() < 18000
    R = gen.euler_zyx(0.3, 1.1, -0.7)
    c = np.array([0.5, -0.2, 0.1])
    inside2 = oracle.surface_inside(V @ R.T + c, T, P @ R.T + c)
    assert np.array_equal(inside2[clear], inside[clear])


def test_ray_parity_fish_surface_matches_its_shape():
    g = gen.fish_ogrid("fish", 64, 48, 8, phase=1.1)
    V, T = gen.body_surface(g)
    rng = np.random.default_rng(4)
    P = np.stack([rng.uniform(-0.55, 0.55, 30000), rng.uniform(-0.2, 0.2, 30000), rng.uniform(-0.12, 0.12, 30000)], 1)
    inside = oracle.surface_inside(V, T, P)
    # compare only points well inside or well outside the analytic body (the facets are chords of it): inside
    # the body shrunk vertically by 1/1.25, or outside it stretched vertically by 1/0.8
    inner = gen.inside_fish_layer(np.stack([P[:, 0], P[:, 1], P[:, 2] * 1.25], 1), 1.1, 0.0)
    outer = ~gen.inside_fish_layer(np.stack([P[:, 0], P[:, 1], P[:, 2] * 0.8], 1), 1.1, 0.0)
    assert inner.sum() > 500 and outer.sum() > 10000
    assert np.all(inside[inner] == 1) and np.all(inside[outer & (np.abs(P[:, 0]) < 0.45)] == 0)


def test_ray_parity_same_along_every_axis():
    """A positive scaling of the axes maps inside to inside, and shrinking one axis 10x makes it the shortest, so
    the ray runs along x, y and z in turn: away from the surface the three answers equal the unscaled one (pins
    the choice of the ray's axis and the order of the projection plane's axes)."""
    g = gen.ellipsoid_ogrid(48, 32, 8, (0.2, 0.1, 0.1), 0.4, beta_r=2.0)
    V, T = gen.body_surface(g)
    rng = np.random.default_rng(9)
    P = rng.uniform(-0.25, 0.25, size=(8000, 3)) * np.array([1.0, 0.6, 0.6])
    f = (P[:, 0] / 0.2) ** 2 + (P[:, 1] / 0.1) ** 2 + (P[:, 2] / 0.1) ** 2
    clear = np.abs(f - 1) > 0.05
    ref = oracle.surface_inside(V, T, P)
    for a in range(3):
        s = np.ones(3)
        s[a] = 0.1
        got = oracle.surface_inside(V * s, T, P * s)
        assert np.array_equal(got[clear], ref[clear]), a
    assert 500 < ref[clear].sum() < clear.sum() - 500


def _torus_surface(R=0.3, r=0.1, nu=64, nv=32):
    """A closed triangulated torus about the z axis (tube radius r, centre radius R)."""
    u = 2 * np.pi * np.arange(nu) / nu
    v = 2 * np.pi * np.arange(nv) / nv
    U, Vv = np.meshgrid(u, v, indexing="ij")
    P = np.stack([(R + r * np.cos(Vv)) * np.cos(U), (R + r * np.cos(Vv)) * np.sin(U), r * np.sin(Vv)], -1)
    V = P.reshape(-1, 3)
    vid = lambda i, j: (i % nu) * nv + (j % nv)
    T = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            T += [(a, b, c), (a, c, d)]
    return V, np.array(T, np.int32)


def test_ray_parity_torus_many_crossings():
    """Rays through a torus cross its surface up to four times: inside iff inside the tube, away from a band
    that covers the facets' chords, with the ray along the torus axis (z is the shortest box axis) and, the z
    axis stretched 5x, across it (x is then the shortest, and rays through the hole cross four times)."""
    R, r = 0.3, 0.1
    V, T = _torus_surface(R, r)
    rng = np.random.default_rng(12)
    P = rng.uniform(-0.45, 0.45, size=(20000, 3)) * np.array([1.0, 1.0, 0.3])
    d = (np.hypot(P[:, 0], P[:, 1]) - R) ** 2 + P[:, 2] ** 2
    clear = np.abs(np.sqrt(d) - r) > 0.01
    want = (d < r * r).astype(np.uint8)
    assert np.array_equal(oracle.surface_inside(V, T, P)[clear], want[clear])
    s = np.array([1.0, 1.0, 5.0])
    assert np.array_equal(oracle.surface_inside(V * s, T, P * s)[clear], want[clear])
    assert 1000 < want[clear].sum() < clear.sum() - 1000


# ----------------------------------------------------------------------------- fluxes at receivers, mass conservation
def _affine_grid(n, A, b, h):
    """Nodes X = b + A (i, j, k) h: every cell a parallelepiped, every face a planar parallelogram."""
    i, j, k = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    ijk = np.stack([i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")], axis=1) * h
    return ijk @ np.asarray(A).T + b


def _curvy_grid(n):
    """A smooth right-handed curvilinear grid on [0,1]^3 (sinusoidal bumps of 0.05 h, zero on the boundary)."""
    g = gen.perturbed_box_grid(n, 1.0, 0.05)
    return g.xyz(), g.dims


def test_flux_of_uniform_field_through_a_closed_surface_is_zero():
    """Half the cross product of the diagonals is the vector area of a quadrilateral (the sum of its edges'
    x_e x x_e+1 / 2); over a closed surface every edge appears twice, reversed, so the areas sum to zero and a
    uniform velocity has no net flux however curved the faces (Sec. 2.4: the flux through a closed surface is zero)."""
    xyz, dims = _curvy_grid(9)
    faces, signs = gen.index_box_surface(dims, (False,) * 3, (1, 2, 1), (7, 6, 8))
    u0 = np.array([0.3, -1.2, 0.7])
    vel = np.tile(u0, (len(xyz), 1))
    U = oracle.face_fluxes(dims, (False,) * 3, xyz, vel, faces)
    assert abs(np.sum(signs * U)) <= 1e-14 * np.sum(np.abs(U))
    # each face on its own: u0 . S with S the face's vector area
    S = np.array([oracle.face_area_vector(xyz, oracle.face_nodes(dims, (False,) * 3, f)) for f in faces])
    assert np.allclose(U, S @ u0, rtol=0, atol=1e-15)


def test_flux_on_affine_grid_matches_closed_forms():
    """On an affine grid (X = b + A ijk h) every face is a parallelogram: its vector area is h^2 (A e_a) x (A e_b)
    and the mean of its corners is its centroid, where a linear field u = G x + u0 takes its face-average value;
    so each flux is exact and the net outward flux of an index box is the divergence times the volume,
    tr(G) det(A) h^3 (number of cells) (divergence theorem).  A wrong diagonal, orientation or sign fails it."""
    rng = np.random.default_rng(21)
    A = np.eye(3) + 0.3 * rng.uniform(-1, 1, (3, 3))
    assert np.linalg.det(A) > 0
    b, h, dims = rng.uniform(-1, 1, 3), 0.1, (7, 6, 8)
    xyz = _affine_grid(dims, A, b, h)
    G = rng.uniform(-1, 1, (3, 3))
    u0 = rng.uniform(-1, 1, 3)
    vel = xyz @ G.T + u0
    lo, hi = (1, 0, 2), (5, 4, 7)
    faces, signs = gen.index_box_surface(dims, (False,) * 3, lo, hi)
    U = oracle.face_fluxes(dims, (False,) * 3, xyz, vel, faces)
    e = np.eye(3)
    for f, Uf in zip(faces, U):
        node, d = divmod(int(f), 3)
        a, bb = (d + 1) % 3, (d + 2) % 3
        S = h * h * np.cross(A @ e[a], A @ e[bb])
        base = np.array([node % dims[0], (node // dims[0]) % dims[1], node // (dims[0] * dims[1])], float)
        centroid = b + A @ ((base + 0.5 * e[a] + 0.5 * e[bb]) * h)
        assert abs(Uf - (G @ centroid + u0) @ S) <= 1e-13
    ncell = np.prod(np.subtract(hi, lo))
    V = np.linalg.det(A) * h ** 3 * ncell
    assert abs(np.sum(signs * U) - np.trace(G) * V) <= 1e-12


def test_mass_correction_removes_the_imbalance_in_proportion_to_area():
    """After the correction the net outward flux of each surface is zero, and every face's flux moved by the same
    amount per unit area, against its outward sign: Delta U_f = -sign_f net |S_f| / sum |S| (Sec. 2.4)."""
    xyz, dims = _curvy_grid(9)
    rng = np.random.default_rng(4)
    vel = rng.uniform(-1, 1, (len(xyz), 3))
    f1, s1 = gen.index_box_surface(dims, (False,) * 3, (0, 0, 0), (4, 5, 3))
    f2, s2 = gen.index_box_surface(dims, (False,) * 3, (3, 2, 4), (8, 8, 8))
    faces, signs = np.concatenate([f1, f2]), np.concatenate([s1, s2])
    start = [0, len(f1), len(faces)]
    U = oracle.face_fluxes(dims, (False,) * 3, xyz, vel, faces)
    Uc, nets, areas = oracle.mass_correct(dims, (False,) * 3, xyz, U, faces, signs, start)
    mag = np.array([np.linalg.norm(oracle.face_area_vector(xyz, oracle.face_nodes(dims, (False,) * 3, f))) for f in faces])
    for s in range(2):
        sl = slice(start[s], start[s + 1])
        assert abs(nets[s] - np.sum(signs[sl] * U[sl])) <= 1e-13
        assert abs(areas[s] - np.sum(mag[sl])) <= 1e-13
        assert abs(np.sum(signs[sl] * Uc[sl])) <= 1e-13 * np.sum(np.abs(U[sl]))
        per_area = (Uc[sl] - U[sl]) * signs[sl] / mag[sl]
        assert np.allclose(per_area, -nets[s] / areas[s], rtol=1e-12, atol=1e-15)
        assert abs(nets[s]) > 1e-3  # a random field really had an imbalance to remove


def test_flux_imbalance_of_a_divergence_free_field_vanishes_with_refinement():
    """A divergence-free field has no net flux through any closed surface; through curved (bilinear) faces the
    corner mean times the vector area misses it by the faces' non-planarity, which shrinks with the cell size:
    on the same smooth grid family (node displacements of 0.1 h along three different sinusoids), halving the
    spacing divides the uncorrected imbalance of a linear and of a quadratic divergence-free field by more than
    four.  (The correction of Sec. 2.4 exists for this imbalance and for that of non-solenoidal intermediate
    velocities.)"""
    G = np.array([[0.4, -1.0, 0.3], [0.8, -0.9, 0.2], [-0.5, 0.6, 0.5]])  # trace 0
    imb = {"linear": [], "quadratic": []}
    for n in (9, 17, 33):
        g = gen.cartesian_grid("c", (n, n, n), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        X, Y, Z = g.x, g.y, g.z
        h = 1.0 / (n - 1)
        xyz = g.xyz() + 0.1 * h * np.stack([np.sin(2 * np.pi * X) * np.sin(3 * np.pi * Y),
                                            np.sin(2 * np.pi * Y) * np.cos(np.pi * Z) * np.sin(np.pi * X),
                                            np.sin(2 * np.pi * Z + 1.0) * X], axis=1)
        q = (n - 1) // 8
        faces, signs = gen.index_box_surface(g.dims, (False,) * 3, (q, 2 * q, q), (7 * q, 6 * q, 8 * q))
        for name, vel in (("linear", xyz @ G.T + np.array([0.1, 0.2, -0.3])),
                          ("quadratic", np.stack([xyz[:, 1] ** 2, xyz[:, 2] ** 2, xyz[:, 0] ** 2], axis=1))):
            U = oracle.face_fluxes(g.dims, (False,) * 3, xyz, vel, faces)
            imb[name].append(abs(np.sum(signs * U)))
    for name, v in imb.items():
        assert v[0] > 1e-8, (name, v)  # curved faces: an imbalance exists
        assert v[0] / v[1] > 4.0 and v[1] / v[2] > 4.0, (name, v)


def test_face_nodes_wrap_on_periodic_axes():
    dims, per = (5, 4, 3), (True, False, False)
    c = oracle.face_nodes(dims, per, 3 * (4 + 5 * (1 + 4 * 0)) + 1)  # base (4,1,0), d = 1: spans k, then i (wraps)
    assert c == [4 + 5 * 1, 4 + 5 * (1 + 4 * 1), 0 + 5 * (1 + 4 * 1), 0 + 5 * 1]
    assert oracle.face_nodes(dims, (False,) * 3, 3 * (4 + 5 * 1) + 1) is None  # leaves a non-periodic grid
