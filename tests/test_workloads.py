"""The seeded synthetic inputs: sizes of the measured configurations, the
Kuhn lattice's geometry, the initial states and the colliders' placement
(the input recipe both the oracle and the CUDA path consume)."""
import numpy as np
import pytest

from paper_1604_07378_gb300 import workloads as W


def _volumes(X, tets):
    d = np.stack([X[tets[:, k]] - X[tets[:, 0]] for k in (1, 2, 3)], axis=-1)
    return np.linalg.det(d) / 6.0


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 4), (5, 1, 2)])
def test_kuhn_lattice_fills_its_box(dims):
    """6 positively oriented tets of volume a^3/6 per cube, filling the box;
    every lattice point is a vertex; every interior face is shared by two
    tets and every boundary face lies on the box."""
    a = 0.05
    X, T = W.kuhn_lattice(*dims, edge=a)
    nx, ny, nz = dims
    assert X.shape == ((nx + 1) * (ny + 1) * (nz + 1), 3) and T.shape == (6 * nx * ny * nz, 4)
    V = _volumes(X, T)
    np.testing.assert_allclose(V, a**3 / 6.0, rtol=1e-12)
    faces = {}
    for t in T:
        for f in ((t[1], t[2], t[3]), (t[0], t[2], t[3]), (t[0], t[1], t[3]), (t[0], t[1], t[2])):
            k = tuple(sorted(int(v) for v in f))
            faces[k] = faces.get(k, 0) + 1
    assert set(faces.values()) <= {1, 2}
    lo, hi = X.min(axis=0), X.max(axis=0)
    for f, c in faces.items():
        if c == 1:  # a boundary face: its three vertices share a box coordinate
            P = X[list(f)]
            assert any(np.all(np.abs(P[:, ax] - b) < 1e-12) for ax in range(3) for b in (lo[ax], hi[ax]))


def test_measured_configurations_sizes():
    w = W.bar_4x4x16_fp64()
    assert (w.n_tets, w.n_verts, int(w.clamped.sum())) == (1536, 425, 25)
    w = W.cube40(W.NEOHOOKEAN)
    assert (w.n_tets, w.n_verts, int(w.clamped.sum())) == (384000, 68921, 1681)
    w = W.spline_bar_80x40x40()
    assert (w.n_tets, w.n_verts) == (768000, 136161)
    w = W.large_48x48x192()
    assert (w.n_tets, w.n_verts) == (2654208, 463393) and (w.iters, w.history) == (20, 8)
    ws = W.batch_512()
    assert len(ws) == 512
    assert sum(x.n_tets for x in ws) == 8747814 and sum(x.n_verts for x in ws) == 1789961
    assert all(4 <= d <= 24 for x in ws for d in x.dims)


def test_cube40_initial_state_is_one_body_velocity():
    """q_l = X; (q_l - q_{l-1}) / h is one velocity drawn from U[-0.5, 0.5]^3
    on every free vertex and zero on the clamped face."""
    w = W.cube40(W.NEOHOOKEAN)
    np.testing.assert_array_equal(w.q_cur, w.rest_pos)
    v = (w.q_cur - w.q_prev) / w.h
    cl = w.clamped.astype(bool)
    assert np.all(v[cl] == 0.0)
    vf = v[~cl]
    np.testing.assert_allclose(vf, np.broadcast_to(vf[0], vf.shape), rtol=0, atol=1e-12)
    assert np.all(np.abs(vf[0]) <= 0.5) and np.any(vf[0] != 0.0)


def test_spline_bar_twist():
    """The initial state turns each cross-section x = const rigidly about the
    bar's axis by 90 deg * x / L; the clamped end x = 0 stays put; the
    initial velocity is zero."""
    w = W.spline_bar_80x40x40(scale=4)
    nx, ny, nz = w.dims
    a = 0.05
    L, yc, zc = nx * a, 0.5 * ny * a, 0.5 * nz * a
    X, q = w.rest_pos, w.q_cur
    np.testing.assert_array_equal(w.q_prev, w.q_cur)
    np.testing.assert_allclose(q[:, 0], X[:, 0], atol=1e-15)
    d0 = (X[:, 1] - yc) + 1j * (X[:, 2] - zc)
    d1 = (q[:, 1] - yc) + 1j * (q[:, 2] - zc)
    np.testing.assert_allclose(np.abs(d1), np.abs(d0), atol=1e-12)
    th = 0.5 * np.pi * X[:, 0] / L
    off = np.abs(d0) > 1e-9
    np.testing.assert_allclose(d1[off] / d0[off], np.exp(1j * th[off]), atol=1e-12)
    cl = w.clamped.astype(bool)
    assert cl.sum() == (ny + 1) * (nz + 1) and np.all(X[cl, 0] == 0.0)
    np.testing.assert_allclose(q[cl], X[cl], atol=1e-15)


@pytest.mark.parametrize("obstacle", ["sphere", "torus"])
def test_collision_drop_obstacle_below_the_cube(obstacle):
    """The unclamped cube starts `drop` above the ground, every vertex moving
    down at `speed`; the obstacle's top is halfway between the ground and the
    cube's lowest face, so nothing penetrates at the start."""
    n, drop, speed = 4, 0.01, 2.0
    w = W.collision_drop(n, drop=drop, speed=speed, torus=(obstacle == "torus"))
    assert not w.clamped.any()
    assert w.q_cur[:, 2].min() == pytest.approx(drop)
    np.testing.assert_allclose((w.q_cur - w.q_prev) / w.h, np.broadcast_to([0.0, 0.0, -speed], w.q_cur.shape),
                               atol=1e-12)
    plane, obs = w.colliders
    assert plane.kind == "plane" and obs.kind == obstacle
    c = np.asarray(obs.point)
    if obstacle == "sphere":
        top = c[2] + obs.radius
        dist = np.linalg.norm(w.q_cur - c, axis=1) - obs.radius
    else:
        assert 0.0 < obs.radius < obs.major
        top = c[2] + obs.radius
        rho = np.linalg.norm(w.q_cur[:, :2] - c[:2], axis=1)
        dist = np.hypot(rho - obs.major, w.q_cur[:, 2] - c[2]) - obs.radius
    assert top == pytest.approx(0.5 * drop)
    assert dist.min() > 0.0
