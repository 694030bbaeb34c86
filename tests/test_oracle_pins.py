"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: hand-derived
closed forms, finite differences, invariances, an independent polar-decomposition
implementation of the projective-dynamics local/global step (Sec. 3-4), the BFGS
secant condition (Alg. 2), exact centre-of-mass motion, and a Newton minimiser.
"""
import json
import math
import os

import types

import numpy as np
import pytest
import scipy.linalg

from oracle import hqn_oracle as O
from paper_1604_07378_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(dims=(2, 2, 3), kind=W.NEOHOOKEAN, E=1e5, nu=0.4, seed=3, v=0.0, clamp=True,
             spline=None, gravity=(0.0, 0.0, -9.81)):
    mat = W.Material(kind, E, nu)
    if kind == W.SPLINE_VL:
        mat.spline = spline if spline is not None else W.spline_control_points(
            mat.mu, mat.lam, np.random.default_rng(seed))
    w = W.lattice_workload(dims, mat, seed=seed, v_range=v, gravity=gravity)
    if not clamp:
        w.clamped[:] = 0
    return w, O.problem_from_workload(w)


MATERIALS = [W.NEOHOOKEAN, W.STVK, W.SPLINE_VL, W.COROTATED, W.POLY4]


# ---------------------------------------------------------------- mesh, mass

def test_kuhn_lattice_volumes_and_mass():
    dims, a = (2, 3, 4), 0.05
    w, P = _problem(dims)
    assert w.n_tets == 6 * 2 * 3 * 4
    assert w.n_verts == 3 * 4 * 5
    np.testing.assert_allclose(P.vol, a**3 / 6.0, rtol=1e-12)
    box = dims[0] * dims[1] * dims[2] * a**3
    assert abs(P.vol.sum() - box) < 1e-12 * box
    assert abs(P.mass.sum() - 1000.0 * box) < 1e-12 * 1000.0 * box
    # every cube's 6 tets cover it: each tet vertex set spans the main diagonal
    t = w.tets.reshape(-1, 6, 4)
    assert np.all(t[:, :, 0] == t[:, :1, 0])


# ---------------------------------------------------------------- signed SVD

def test_signed_svd_convention():
    rng = np.random.default_rng(0)
    F = rng.normal(size=(2000, 3, 3))
    F[:1000] += 2.0 * np.eye(3)
    U, s, V = O.signed_svd(F)
    rec = U @ (s[:, :, None] * np.swapaxes(V, -1, -2))
    assert np.max(np.abs(rec - F)) < 1e-12 * np.max(np.abs(F))
    np.testing.assert_allclose(np.linalg.det(U), 1.0, atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(V), 1.0, atol=1e-12)
    assert np.all(s[:, 0] >= s[:, 1] - 1e-14) and np.all(s[:, 1] >= np.abs(s[:, 2]) - 1e-14)
    assert np.all(np.sign(s[:, 2]) == np.sign(np.linalg.det(F)))
    # reflection through one axis: stretches (3, 2, -1)
    _, s1, _ = O.signed_svd(np.diag([3.0, -2.0, 1.0])[None])
    np.testing.assert_allclose(s1[0], [3.0, 2.0, -1.0], atol=1e-14)
    # a rotation: unit stretches and U V^T = R
    R = scipy.linalg.expm(np.array([[0, -0.3, 0.2], [0.3, 0, -0.7], [-0.2, 0.7, 0]]))
    U, s2, V = O.signed_svd(R[None])
    np.testing.assert_allclose(s2[0], 1.0, atol=1e-14)
    np.testing.assert_allclose(U[0] @ V[0].T, R, atol=1e-14)


# ---------------------------------------------------------------- materials

def _random_F(rng, n, spread=0.3, allow_inverted=False):
    F = np.eye(3) + spread * rng.normal(size=(n, 3, 3))
    if not allow_inverted:
        F[np.linalg.det(F) < 0.2] = np.eye(3)
    return F


def test_neohookean_matches_invariant_form():
    mu, lam = O.lame(1e5, 0.45)
    mat = O.NeoHookean(mu, lam)
    F = _random_F(np.random.default_rng(1), 500)
    _, s, _ = O.signed_svd(F)
    J = np.linalg.det(F)
    I1 = np.einsum("nij,nij->n", F, F)
    ref = 0.5 * mu * (I1 - 3.0) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2
    np.testing.assert_allclose(O.psi(mat, s), ref, rtol=1e-11, atol=1e-9 * mu)


def test_stvk_matches_invariant_form():
    mu, lam = O.lame(5e5, 0.4)
    mat = O.StVK(mu, lam)
    F = _random_F(np.random.default_rng(2), 500, allow_inverted=True)
    _, s, _ = O.signed_svd(F)
    Eg = 0.5 * (np.swapaxes(F, -1, -2) @ F - np.eye(3))
    ref = mu * np.einsum("nij,nij->n", Eg, Eg) + 0.5 * lam * np.trace(Eg, axis1=1, axis2=2) ** 2
    np.testing.assert_allclose(O.psi(mat, s), ref, rtol=1e-11, atol=1e-9 * mu)


def test_corotated_and_poly4_match_polar_forms():
    mu, lam = 20.0, 100.0
    F = _random_F(np.random.default_rng(3), 300)
    _, s, _ = O.signed_svd(F)
    R = np.stack([scipy.linalg.polar(f)[0] for f in F])
    J = np.linalg.det(F)
    ref = mu * np.einsum("nij,nij->n", F - R, F - R) + 0.5 * lam * (J - 1.0) ** 2
    np.testing.assert_allclose(O.psi(O.Corotated(mu, lam), s), ref, rtol=1e-10, atol=1e-12)
    ev = np.sqrt(np.linalg.eigvalsh(np.swapaxes(F, -1, -2) @ F))
    np.testing.assert_allclose(O.psi(O.Poly4(mu), s), mu * np.sum((ev - 1.0) ** 4, axis=1),
                               rtol=1e-10, atol=1e-12)


def test_spline_reproduces_quadratic_material_exactly():
    """Cubic Hermite splines sampling a quadratic reproduce it everywhere,
    including the quadratic extension outside the knots."""
    mu, lam = 7.0, 11.0
    k = np.asarray(W.SPLINE_KNOTS)
    ctrl = np.zeros((3, k.size, 3))
    ctrl[:, :, 0] = k
    ctrl[0, :, 1], ctrl[0, :, 2] = mu * (k - 1) ** 2, 2 * mu * (k - 1)
    ctrl[2, :, 1], ctrl[2, :, 2] = 0.5 * lam * (k - 1) ** 2, lam * (k - 1)
    spl, cor = O.SplineVL(ctrl), O.Corotated(mu, lam)
    t = np.linspace(-0.5, 4.0, 301)
    for f in ("a", "da", "b", "db", "c", "dc"):
        np.testing.assert_allclose(getattr(spl, f)(t), getattr(cor, f)(t), atol=1e-11)
    assert abs(O.stiffness_k(spl) - (2 * mu + lam)) < 1e-10 * (2 * mu + lam)


# ---------------------------------------------------------------- stiffness k (Eq. stiffness)

def test_stiffness_closed_forms():
    """k = 12 * integral_{1/2}^{3/2} (s - 1) f(s) ds, derived by hand per material."""
    mu, lam = O.lame(5e5, 0.4)
    k_cor = 2 * mu + lam
    k_poly = 0.6 * mu
    F = lambda s: s * math.log(s) - s - 0.5 * math.log(s) ** 2
    k_nh = mu * (12.0 * math.log(3.0) - 11.0) + lam * 12.0 * (F(1.5) - F(0.5))
    k_stvk = 2.15 * (mu + 0.5 * lam)              # 12 * 43/240 = 43/20
    assert abs(O.stiffness_k(O.Corotated(mu, lam)) - k_cor) < 1e-10 * k_cor
    assert abs(O.stiffness_k(O.Poly4(mu)) - k_poly) < 1e-10 * k_poly
    assert abs(O.stiffness_k(O.NeoHookean(mu, lam)) - k_nh) < 1e-10 * k_nh
    assert abs(O.stiffness_k(O.StVK(mu, lam)) - k_stvk) < 1e-10 * k_stvk
    # the paper: for the polynomial material k depends linearly on mu
    assert abs(O.stiffness_k(O.Poly4(3 * mu)) - 3 * k_poly) < 1e-9 * k_poly


def test_stiffness_spline_matches_brute_force_integral():
    """Eq. stiffness for a spline material, whose integrand is only piecewise
    smooth: the oracle's k equals the defining integral ratio evaluated by a
    composite midpoint rule on 2e6 cells (error O(h^2) ~ 1e-12 per piece)."""
    mu, lam = O.lame(5e5, 0.4)
    ctrl = W.spline_control_points(mu, lam, np.random.default_rng(1606))
    mat = O.SplineVL(ctrl)
    n = 2_000_000
    s = 0.5 + (np.arange(n) + 0.5) / n
    f = mat.da(s) + 2.0 * mat.db(s) + mat.dc(s)
    k_brute = np.sum((s - 1.0) * f) / n / (1.0 / 12.0)
    assert abs(O.stiffness_k(mat) - k_brute) < 1e-9 * abs(k_brute)


def test_paper_parameters_golden():
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as f:
        g = json.load(f)
    assert g["h"] == pytest.approx(1.0 / 30.0)
    assert (g["x_start"], g["x_end"]) == (0.5, 1.5)
    w = W.cube40(n=2)
    assert w.h == pytest.approx(g["h"]) and w.history == g["history_m"] and w.iters == g["iterations"]
    # the oracle's defaults are the paper's
    import inspect
    sig = inspect.signature(O.solve_step).parameters
    assert sig["gamma"].default == g["gamma"] and sig["backtrack"].default == g["backtrack"]
    assert sig["m"].default == g["history_m"] and sig["iters"].default == g["iterations"]


# ---------------------------------------------------------------- gradient of g

@pytest.mark.parametrize("kind", MATERIALS)
def test_gradient_matches_central_differences(kind):
    w, P = _problem((2, 2, 3), kind=kind, seed=5)
    rng = np.random.default_rng(11)
    x = w.rest_pos + 0.012 * rng.normal(size=w.rest_pos.shape)
    y = w.rest_pos + 0.01 * rng.normal(size=w.rest_pos.shape)
    x[P.clamped] = w.rest_pos[P.clamped]
    y[P.clamped] = w.rest_pos[P.clamped]
    if kind == W.NEOHOOKEAN:
        # push one vertex through its neighbours: inverted tets use the J < J0 extension
        v = P.free[len(P.free) // 2]
        x[v] += np.array([0.06, 0.05, -0.055])
        J = np.linalg.det(O.deformation_gradients(P, x))
        assert np.any(J < 0.0) and np.any(J > O.J0_NEOHOOKEAN)
    grad = O.gradient(P, x, y)
    eps = 1e-7
    fd = np.zeros_like(x)
    for v in P.free:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += eps
            xm[v, c] -= eps
            fd[v, c] = (O.objective(P, xp, y) - O.objective(P, xm, y)) / (2 * eps)
    err = np.linalg.norm(fd - grad) / np.linalg.norm(grad)
    assert err < 1e-6, err
    assert np.all(grad[P.clamped] == 0.0)


@pytest.mark.parametrize("kind", MATERIALS)
def test_zero_force_and_energy_at_rest(kind):
    w, P = _problem((2, 2, 3), kind=kind)
    X = w.rest_pos
    grad = O.gradient(P, X, X)
    scale = P.k * 0.05**2
    assert np.max(np.abs(grad)) < 1e-9 * scale
    assert abs(O.objective(P, X, X)) < 1e-12 * scale * 0.05


@pytest.mark.parametrize("kind", MATERIALS)
def test_energy_rotation_translation_invariance(kind):
    w, P = _problem((2, 2, 2), kind=kind)
    rng = np.random.default_rng(7)
    x = w.rest_pos + 0.01 * rng.normal(size=w.rest_pos.shape)
    R = scipy.linalg.expm(np.array([[0, -1.1, 0.4], [1.1, 0, -0.9], [-0.4, 0.9, 0]]))
    x2 = x @ R.T + np.array([0.3, -2.0, 5.0])
    e1 = np.sum(O.elastic_energy_per_tet(P, x))
    e2 = np.sum(O.elastic_energy_per_tet(P, x2))
    assert abs(e1 - e2) < 1e-10 * abs(e1)


# ---------------------------------------------------------------- A0 = M/h^2 + L

def test_A0_spd_residual_and_laplacian():
    w, P = _problem((3, 2, 4))
    A = P.A.toarray()
    assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    np.linalg.cholesky(A)                                   # SPD
    rng = np.random.default_rng(1)
    q = rng.normal(size=(P.n, 3))
    q[P.clamped] = 0.0
    r = O.solve_A(P, q)
    res = P.A @ r[P.free] - q[P.free]
    assert np.linalg.norm(res) < 1e-12 * np.linalg.norm(q)
    # constants are in the null space of every G_t
    L = O.laplacian(P)
    assert np.max(np.abs(L @ np.ones(P.n))) < 1e-10 * np.abs(L).max()
    # x^T L x = sum_t w_t ||G_t x||_F^2 with G_t x = F(x)^T built from Ds Dm^{-1}
    x = rng.normal(size=(P.n, 3))
    Fx = O.deformation_gradients(P, x)
    lhs = np.sum(x * (L @ x))
    rhs = np.sum(P.vol * P.k * np.einsum("tij,tij->t", Fx, Fx))
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)


# ---------------------------------------------------------------- Alg. 2

def test_two_loop_m0_is_alg1_direction():
    w, P = _problem((2, 2, 3), seed=2, v=0.3)
    y = O.predictor(P, w.q_cur, w.q_prev)
    grad = O.gradient(P, y + 0.003, y)
    d = O.lbfgs_direction(P, grad, [])
    np.testing.assert_allclose(d, -O.solve_A(P, grad), rtol=0, atol=1e-15)


def test_two_loop_secant_condition_and_symmetry():
    """The L-BFGS inverse-Hessian operator B satisfies B t_newest = s_newest and
    is symmetric (Nocedal-Wright Ch. 7); d = -B grad in Alg. 2."""
    w, P = _problem((2, 2, 3), seed=4)
    rng = np.random.default_rng(9)
    nf = P.free.size
    Q = rng.normal(size=(3 * nf, 3 * nf))
    H = Q @ Q.T + 3 * nf * np.eye(3 * nf)
    hist = []
    for _ in range(4):
        s = np.zeros((P.n, 3))
        s[P.free] = rng.normal(size=(nf, 3))
        t = np.zeros((P.n, 3))
        t[P.free] = (H @ s[P.free].ravel()).reshape(nf, 3)
        hist.append((s, t, O.tr_dot(t, s)))
    s_new, t_new, _ = hist[-1]
    d = O.lbfgs_direction(P, -t_new, hist)
    assert np.linalg.norm(d - s_new) < 1e-10 * np.linalg.norm(s_new)
    u = np.zeros((P.n, 3)); u[P.free] = rng.normal(size=(nf, 3))
    v = np.zeros((P.n, 3)); v[P.free] = rng.normal(size=(nf, 3))
    Bu = -O.lbfgs_direction(P, u, hist)
    Bv = -O.lbfgs_direction(P, v, hist)
    assert abs(O.tr_dot(v, Bu) - O.tr_dot(u, Bv)) < 1e-10 * abs(O.tr_dot(v, Bu))
    assert O.tr_dot(u, Bu) > 0


# ---------------------------------------------------------------- Sec. 4: projective dynamics

def test_projective_dynamics_identity_arap():
    """For ARAP (corotated, lam = 0) the energy is a projective-dynamics energy
    with w = V k, k = 2 mu.  Then d = x* - x where x* is the local/global step
    (Eq. PDsolution), built here from polar projections, and alpha = 1 always
    passes the Armijo test with gamma = 0.3."""
    w, P = _problem((2, 2, 4), kind=W.COROTATED, E=2e4, nu=0.0, v=0.4, seed=8)
    assert abs(P.k - 2 * P.mat.mu) < 1e-10 * P.k
    y = O.predictor(P, w.q_cur, w.q_prev)
    x = y.copy()
    rng = np.random.default_rng(5)
    x[P.free] += 0.004 * rng.normal(size=(P.free.size, 3))
    d = O.lbfgs_direction(P, O.gradient(P, x, y), [])
    # independent local step: p_t = polar rotation of F_t; residual of the global step
    Fx = O.deformation_gradients(P, x)
    res = P.mass[:, None] * (x - y) / P.h**2
    B = np.array([[-1.0, 1.0, 0.0, 0.0], [-1.0, 0.0, 1.0, 0.0], [-1.0, 0.0, 0.0, 1.0]])
    for t in range(P.tets.shape[0]):
        R = scipy.linalg.polar(Fx[t])[0]
        Gt = P.Dm_inv[t].T @ B                       # 3 x 4
        contrib = P.vol[t] * P.k * Gt.T @ (Fx[t].T - R.T)   # 4 x 3
        for c in range(4):
            res[P.tets[t, c]] += contrib[c]
    delta = np.zeros_like(x)
    delta[P.free] = np.linalg.solve(P.A.toarray(), -res[P.free])
    assert np.linalg.norm(delta - d) < 1e-9 * np.linalg.norm(d)
    _, st = O.solve_step(P, w.q_cur, w.q_prev, iters=10, m=0)
    assert st.trials == [1] * 10


# ---------------------------------------------------------------- whole step

def test_centre_of_mass_follows_ballistic_motion():
    """Unclamped body: elastic forces sum to zero and 1^T L = 0, so every iterate
    keeps sum_v m_v x_v = sum_v m_v y_v (Eq. PD with y = 2q_l - q_{l-1} + h^2 g)."""
    w, P = _problem((2, 3, 3), kind=W.STVK, v=0.6, seed=12, clamp=False)
    x, st = O.solve_step(P, w.q_cur, w.q_prev, iters=10, m=5)
    M = P.mass.sum()
    com = (P.mass[:, None] * x).sum(0) / M
    com_ref = (P.mass[:, None] * (2 * w.q_cur - w.q_prev)).sum(0) / M + P.h**2 * np.array(w.gravity)
    assert np.linalg.norm(com - com_ref) < 1e-12 * np.linalg.norm(com_ref)
    assert st.g[-1] < st.g0


@pytest.mark.parametrize("dims,kind", [((1, 1, 2), W.NEOHOOKEAN), ((2, 2, 3), W.STVK)])
def test_converged_lbfgs_equals_newton_minimiser(dims, kind):
    w, P = _problem(dims, kind=kind, v=0.8, seed=21)
    x_newton, g_newton = O.newton_minimise(P, w.q_cur, w.q_prev)
    x_lbfgs, st = O.solve_step(P, w.q_cur, w.q_prev, iters=300, m=5)
    y = O.predictor(P, w.q_cur, w.q_prev)
    scale = np.linalg.norm(x_newton - y)
    assert scale > 1e-4
    assert np.linalg.norm(x_lbfgs - x_newton) < 1e-6 * scale
    assert abs(st.g[-1] - g_newton) <= 1e-10 * abs(st.g0 - g_newton)


def test_lbfgs_history_speeds_convergence():
    """Sec. 5: L-BFGS (m = 5) reaches a lower relative error (Eq. RelativeError)
    than the plain quasi-Newton direction (m = 0) after 10 iterations."""
    w = W.spline_bar_80x40x40(scale=10)
    w.material = W.Material(W.NEOHOOKEAN, 5e5, 0.4)
    P = O.problem_from_workload(w)
    _, st_ref = O.solve_step(P, w.q_cur, w.q_prev, iters=400, m=5)
    g_star = st_ref.g[-1]
    _, st0 = O.solve_step(P, w.q_cur, w.q_prev, iters=10, m=0)
    _, st5 = O.solve_step(P, w.q_cur, w.q_prev, iters=10, m=5)
    e0 = O.relative_error(st0.g[-1], st0.g0, g_star)
    e5 = O.relative_error(st5.g[-1], st5.g0, g_star)
    assert 0 <= e5 < e0 < 1


# ---------------------------------------------------------------- collisions (Sec. 4.3)

def _drop_problem(n=3, **kw):
    w = W.collision_drop(n, **kw)
    return w, O.problem_from_workload(w)


def test_contact_gradient_matches_central_differences():
    """The collision terms' gradient is the derivative of their energy (the
    active set and the frozen t, n held fixed), on top of the elastic and
    inertia terms."""
    w, P = _drop_problem(3, drop=-0.01, speed=1.0)
    y = O.predictor(P, w.q_cur, w.q_prev)
    rng = np.random.default_rng(3)
    x = y + 1e-3 * rng.normal(size=y.shape)
    C = O.contact_terms(P, x, w.q_cur)
    assert C.idx.size > 0
    g = O.gradient(P, x, y, C)
    eps = 1e-6
    for v in C.idx[:4]:
        for c in range(3):
            xp = x.copy(); xp[v, c] += eps
            xm = x.copy(); xm[v, c] -= eps
            fd = (O.objective(P, xp, y, C) - O.objective(P, xm, y, C)) / (2 * eps)
            assert abs(fd - g[v, c]) <= 1e-6 * max(1.0, abs(g[v, c])), (v, c, fd, g[v, c])


def test_contact_set_penetrating_and_approaching_only():
    """A vertex below the plane is active only if it is not moving away; a
    vertex above the plane never is; the surface point is the vertex's
    projection and the normal the plane's."""
    w, P = _drop_problem(2, sphere=False)
    x = w.rest_pos.copy()
    q_ref = x.copy()
    x[:, 2] += 0.01           # everything above z = 0 ...
    x[0, 2] = -0.004          # ... but vertex 0 (moving down from 0)
    x[1, 2] = -0.002          # and vertex 1, which moves up into the plane
    q_ref[1, 2] = -0.003
    C = O.contact_terms(P, x, q_ref)
    assert list(C.idx) == [0]
    np.testing.assert_allclose(C.t[0], [x[0, 0], x[0, 1], 0.0], atol=1e-15)
    np.testing.assert_allclose(C.n[0], [0.0, 0.0, 1.0])
    assert C.w[0] == pytest.approx(P.contact_scale * P.mass[0] / P.h**2)
    assert O.contact_energy(C, x) == pytest.approx(C.w[0] * 0.004**2)


def test_sphere_contact_projection():
    w, P = _drop_problem(2)
    cen, r = np.asarray(w.colliders[1].point), w.colliders[1].radius
    x = w.rest_pos.copy() + 5.0  # far away ...
    d = np.array([1.0, 2.0, 2.0]) / 3.0
    x[3] = cen + 0.9 * r * d      # ... except vertex 3, inside the sphere
    C = O.contact_terms(P, x, x + 0.01 * d)   # moved inwards over the step
    assert list(C.idx) == [3]
    np.testing.assert_allclose(C.n[0], d, atol=1e-14)
    np.testing.assert_allclose(C.t[0], cen + r * d, atol=1e-14)


def test_drop_onto_colliders_is_stopped():
    """The falling cube is stopped by the ground: over 15 steps no vertex
    sinks more than 1 cm below z = 0 and the centre of mass, falling at 2 m/s,
    has stopped falling; every step keeps the objective below g(x_1)."""
    w, P = _drop_problem(3, drop=0.005, speed=2.0)
    qc, qp = w.q_cur.copy(), w.q_prev.copy()
    for _ in range(15):
        x, st = O.solve_step(P, qc, qp, iters=10, m=5)
        assert not st.exhausted
        assert min(st.g) < st.g0
        assert x[:, 2].min() > -0.01
        qp, qc = qc, x
    vz = (qc[:, 2] - qp[:, 2]).mean() / P.h
    assert vz > -0.3, vz


# ---------------------------------------------------------------- anisotropic fibre term (Sec. 4.4)

def test_fiber_term_closed_form_and_invariances():
    """kappa/2 (|F d| - 1)^2 per unit volume: a stretch s along d adds exactly
    V kappa/2 (s - 1)^2 to the base energy, a stretch across d adds nothing,
    the term vanishes at rest and is invariant under rotations of the
    deformed state; the stiffness fit keeps the base material's k."""
    w = W.fiber_cube(2, fiber=(1.0, 0.0, 0.0))
    P = O.problem_from_workload(w)
    base = O.problem_from_workload(W.lattice_workload((2, 2, 2), w.material.__class__(
        w.material.kind, w.material.E, w.material.nu), clamp_axis=2))
    assert P.k == base.k
    X = w.rest_pos
    assert np.allclose(O.elastic_energy_per_tet(P, X), 0.0)
    for s, axis, extra in ((1.3, 0, True), (0.8, 0, True), (1.3, 1, False)):
        x = X.copy()
        x[:, axis] *= s
        e = O.elastic_energy_per_tet(P, x) - O.elastic_energy_per_tet(base, x)
        expect = P.vol * 0.5 * P.mat.kappa * (s - 1.0) ** 2 if extra else 0.0 * P.vol
        np.testing.assert_allclose(e, expect, rtol=1e-12, atol=1e-9 * np.abs(expect).max() if extra else 1e-9)
    rng = np.random.default_rng(2)
    x = X + 0.01 * rng.normal(size=X.shape)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Q *= np.sign(np.linalg.det(Q))
    np.testing.assert_allclose(O.elastic_energy_per_tet(P, x @ Q.T), O.elastic_energy_per_tet(P, x), rtol=1e-10)


def test_fiber_gradient_matches_central_differences():
    w = W.fiber_cube(2)
    P = O.problem_from_workload(w)
    rng = np.random.default_rng(12)
    x = w.rest_pos + 0.01 * rng.normal(size=w.rest_pos.shape)
    y = w.rest_pos + 0.01 * rng.normal(size=w.rest_pos.shape)
    x[P.clamped] = w.rest_pos[P.clamped]
    y[P.clamped] = w.rest_pos[P.clamped]
    grad = O.gradient(P, x, y)
    eps = 1e-7
    fd = np.zeros_like(x)
    for v in P.free:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += eps
            xm[v, c] -= eps
            fd[v, c] = (O.objective(P, xp, y) - O.objective(P, xm, y)) / (2 * eps)
    assert np.linalg.norm(fd - grad) / np.linalg.norm(grad) < 1e-6


# ---------------------------------------------------------------- Jacobi-PCG in lieu of A0^{-1} (Sec. 8)

def test_pcg_is_conjugate_gradients_and_converges():
    """The fixed-iteration Jacobi-PCG equals the textbook method: one
    iteration is the preconditioned steepest-descent step with the exact line
    minimiser; enough iterations reach A0^{-1} q; the error in the A0 norm
    never grows; and scipy's CG with the same preconditioner agrees."""
    import scipy.sparse.linalg as spla
    w, P = _problem((3, 3, 4), kind=W.NEOHOOKEAN, seed=8)
    rng = np.random.default_rng(4)
    q = rng.normal(size=(P.n, 3))
    q[P.clamped] = 0.0
    exact = O.solve_A(P, q)
    b = q[P.free]
    dinv = 1.0 / O.jacobi_diagonal(P)
    z = dinv[:, None] * b
    alpha = O.tr_dot(b, z) / O.tr_dot(z, P.A @ z)
    np.testing.assert_allclose(O.solve_A_pcg(P, q, 1)[P.free], alpha * z, rtol=1e-12)
    errs = []
    for k in (1, 2, 5, 15, 60):
        e = (O.solve_A_pcg(P, q, k) - exact)[P.free]
        errs.append(np.sqrt(O.tr_dot(e, P.A @ e)))
    assert all(b2 <= b1 * (1 + 1e-12) for b1, b2 in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-10 * errs[0]
    # column by column, scipy's CG sees a different (per-column) step length:
    # compare on a single right-hand side, where the two coincide
    q1 = np.zeros_like(q)
    q1[:, 0] = q[:, 0]
    ours = O.solve_A_pcg(P, q1, 7)[P.free, 0]
    M = spla.LinearOperator(P.A.shape, matvec=lambda v: dinv * v)
    ref, _ = spla.cg(P.A, q1[P.free, 0], x0=np.zeros(P.free.size), rtol=0.0, atol=0.0, maxiter=7, M=M)
    np.testing.assert_allclose(ours, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_pcg_step_runs_and_decreases_objective():
    """Alg. 1 with 15 Jacobi-PCG iterations in lieu of the factorised A0:
    every iteration decreases g, and the result is close to the direct-solve
    step (the paper reports competitive convergence)."""
    w, P = _problem((3, 3, 6), kind=W.NEOHOOKEAN, seed=9)
    x_d, st_d = O.solve_step(P, w.q_cur, w.q_prev)
    x_p, st_p = O.solve_step(P, w.q_cur, w.q_prev, pcg_iters=15)
    gs = [st_p.g0] + st_p.g
    assert all(b < a for a, b in zip(gs, gs[1:]))
    assert np.linalg.norm(x_p - x_d) / np.linalg.norm(x_d) < 1e-3


# ---------------------------------------------------------------- Chebyshev direction (Alg. 3) and Eq. RelativeError

def test_chebyshev_weights_and_pd_limit():
    """omega_{k+1} follows Alg. 3 and tends to the Chebyshev fixed point
    2 / (1 + sqrt(1 - rho^2)); while omega = 1 (k < S) the direction is the
    projective-dynamics one, -A0^{-1} grad (L-BFGS with m = 0)."""
    rho, S = 0.95, 10
    om = 1.0
    for k in range(1, 200):
        om = O.chebyshev_omega(k, S, rho, om)
        if k < S:
            assert om == 1.0
        if k == S:
            assert om == pytest.approx(2.0 / (2.0 - rho * rho))
    assert om == pytest.approx(2.0 / (1.0 + math.sqrt(1.0 - rho * rho)), rel=1e-12)
    w = W.spline_bar_80x40x40(scale=10)
    P = O.problem_from_workload(w)
    x_c, st_c = O.solve_step(P, w.q_cur, w.q_prev, iters=8, chebyshev=(S, rho))
    x_p, st_p = O.solve_step(P, w.q_cur, w.q_prev, iters=8, m=0)
    np.testing.assert_allclose(x_c, x_p, rtol=0, atol=1e-12 * np.abs(x_p).max())
    assert st_c.trials == st_p.trials


def test_relative_error_ordering_on_twisted_bar():
    """Eq. RelativeError on the twisting spline bar, x* from a long L-BFGS
    run: after 40 iterations Chebyshev (S = 10, rho = 0.99) beats projective
    dynamics (m = 0) and L-BFGS with m = 5 beats both -- the ordering of the
    paper's comparison of methods."""
    w = W.spline_bar_80x40x40(scale=10)
    P = O.problem_from_workload(w)
    _, st_star = O.solve_step(P, w.q_cur, w.q_prev, iters=300, m=8)
    g_star = min(st_star.g)
    err = {}
    for name, kw in (("pd", dict(m=0)), ("cheb", dict(m=0, chebyshev=(10, 0.99))), ("lbfgs5", dict(m=5))):
        _, st = O.solve_step(P, w.q_cur, w.q_prev, iters=40, **kw)
        err[name] = O.relative_error(st.g[-1], st.g0, g_star)
    assert 0.0 <= err["lbfgs5"] < err["cheb"] < err["pd"] < 1.0, err


def _torus_surface_distance(x, c, a, R, r, n_theta=720, n_phi=360):
    """Brute force: the distance from x to a dense sampling of the torus
    surface c + (R + r cos phi) e(theta) + r sin phi a."""
    a = np.asarray(a, float) / np.linalg.norm(a)
    e1 = np.cross(a, [1.0, 0.0, 0.0])
    if np.linalg.norm(e1) < 1e-6:
        e1 = np.cross(a, [0.0, 1.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    th = np.linspace(0.0, 2 * np.pi, n_theta, endpoint=False)
    ph = np.linspace(0.0, 2 * np.pi, n_phi, endpoint=False)
    T, Ph = np.meshgrid(th, ph, indexing="ij")
    ring = np.cos(T)[..., None] * e1 + np.sin(T)[..., None] * e2
    pts = c + (R + r * np.cos(Ph))[..., None] * ring + (r * np.sin(Ph))[..., None] * a
    d = np.linalg.norm(pts.reshape(-1, 3) - x, axis=1)
    k = int(np.argmin(d))
    return d[k], pts.reshape(-1, 3)[k]


def test_torus_contact_projection_against_brute_force():
    """For points inside the tube of a tilted torus, the surface point t is
    the nearest point of the surface (brute force over a dense (theta, phi)
    grid), |x - t| = -phi, n is the unit vector from t towards the tube's
    centre circle's outside, and points outside the tube, on the axis or in
    the hole are not in contact."""
    c, a, R, r = np.array([0.1, -0.2, 0.3]), np.array([1.0, 2.0, 2.0]) / 3.0, 0.5, 0.15
    col = ("torus", tuple(c), tuple(a), R, r)
    e1 = np.cross(a, [1.0, 0.0, 0.0]); e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    rng = np.random.default_rng(17)
    pts = []
    for _ in range(6):  # inside the tube at random angles and depths
        th, ph, rr = rng.uniform(0, 2 * np.pi), rng.uniform(0, 2 * np.pi), rng.uniform(0.2, 0.9) * r
        ring = np.cos(th) * e1 + np.sin(th) * e2
        pts.append(c + (R + rr * np.cos(ph)) * ring + rr * np.sin(ph) * a)
    pts.append(c + (R + 1.5 * r) * e1)      # outside the tube
    pts.append(c + 0.3 * a)                  # on the axis (in the hole)
    pts.append(c + 0.5 * (R - r) * e2)       # in the hole, off the axis
    x = np.array(pts)
    # contact_terms reads only these fields of a problem
    P = types.SimpleNamespace(n=x.shape[0], free=np.arange(x.shape[0]), colliders=(col,),
                              contact_scale=1.0, mass=np.ones(x.shape[0]), h=1.0)
    C = O.contact_terms(P, x, x)   # not moving: vn = 0 keeps every penetrating vertex
    assert list(C.idx) == list(range(6))
    for k, v in enumerate(C.idx):
        d_bf, p_bf = _torus_surface_distance(x[v], c, a, R, r)
        depth = np.linalg.norm(x[v] - C.t[k])
        assert abs(depth - d_bf) <= 2e-3 * r, (depth, d_bf)
        assert np.linalg.norm(C.t[k] - p_bf) <= 0.02 * r
        assert abs(np.linalg.norm(C.n[k]) - 1.0) <= 1e-14
        # x lies on the inward side: x = t - depth n
        np.testing.assert_allclose(x[v], C.t[k] - depth * C.n[k], atol=1e-14)


def test_torus_contact_gradient_matches_central_differences():
    """The cube dropped onto the ring, one step after the first contact: the
    torus terms' gradient is the derivative of their energy."""
    w = W.collision_drop(4, drop=0.004, speed=2.0, torus=True)
    P = O.problem_from_workload(w)
    qc, _ = O.solve_step(P, w.q_cur, w.q_prev, iters=10, m=5)
    qp = w.q_cur
    y = O.predictor(P, qc, qp)
    rng = np.random.default_rng(5)
    x = y + 1e-4 * rng.normal(size=y.shape)
    C = O.contact_terms(P, x, qc)
    tor = [k for k in range(C.idx.size) if abs(C.n[k, 2]) < 0.999]  # normals off the plane's
    assert len(tor) > 0
    g = O.gradient(P, x, y, C)
    eps = 1e-6
    for k in tor[:3]:
        v = C.idx[k]
        for cc in range(3):
            xp = x.copy(); xp[v, cc] += eps
            xm = x.copy(); xm[v, cc] -= eps
            fd = (O.objective(P, xp, y, C) - O.objective(P, xm, y, C)) / (2 * eps)
            assert abs(fd - g[v, cc]) <= 1e-6 * max(1.0, abs(g[v, cc])), (v, cc, fd, g[v, cc])


def test_A0_quadratic_form_of_an_affine_displacement():
    """Closed form of Eq. PDmatrixForm's quadratic form: for an affine
    displacement u_v = B X_v every tet has F - I = B, so on an unclamped mesh
    u^T A0 u = sum_v m_v |u_v|^2 / h^2 + k V_total |B|_F^2 (the three
    coordinates summed); with the lumped masses m_v = rho sum_{t∋v} V_t / 4
    counted by brute force over the tets.  A transposed gradient operator,
    a missing volume or stiffness factor, or a wrong mass fails it."""
    w = W.lattice_workload((3, 2, 4), W.Material(W.NEOHOOKEAN, 3e5, 0.35), clamp_axis=-1)
    P = O.problem_from_workload(w)
    A = O.assemble_A(P)
    assert A.shape == (w.n_verts, w.n_verts)
    rng = np.random.default_rng(23)
    B = rng.normal(size=(3, 3))
    u = w.rest_pos @ B.T
    quad = sum(float(u[:, c] @ (A @ u[:, c])) for c in range(3))
    vols = []
    for t in w.tets:
        X0, X1, X2, X3 = w.rest_pos[t]
        vols.append(np.linalg.det(np.column_stack([X1 - X0, X2 - X0, X3 - X0])) / 6.0)
    vols = np.array(vols)
    m = np.zeros(w.n_verts)
    for t, V in zip(w.tets, vols):
        m[t] += w.material.density * V / 4.0
    expect = float(np.sum(m * np.sum(u * u, axis=1))) / w.h**2 + P.k * vols.sum() * float(np.sum(B * B))
    assert quad == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("npairs,dims", [(7, (2, 2, 3)), (100, (3, 3, 4))], ids=["7", "100"])
def test_two_loop_equals_dense_bfgs_with_full_memory(npairs, dims):
    """With every pair kept (memory at least the pairs, e.g. the paper's
    m = 100 study), Alg. 2's two-loop recursion applies exactly the BFGS
    inverse Hessian built by the textbook dense update, started from
    H0 = A0^{-1} (the same on the x, y and z columns):
    H <- (I - r s t^T) H (I - r t s^T) + r s s^T, r = 1 / t^T s, oldest pair
    first (Nocedal-Wright eq. 6.17).  A pair applied in the wrong order or
    with the wrong scaling fails it (the 100 pairs applied newest first
    differ by 38%); 100 pairs on 192 unknowns is the paper's longest window
    (the two forms agree to ~1e-14)."""
    w, P = _problem(dims, seed=6)
    rng = np.random.default_rng(31)
    nf = P.free.size
    Q = rng.normal(size=(3 * nf, 3 * nf))
    Htrue = Q @ Q.T + 3 * nf * np.eye(3 * nf)
    hist, pairs = [], []
    for _ in range(npairs):
        s = np.zeros((P.n, 3))
        s[P.free] = rng.normal(size=(nf, 3))
        t = np.zeros((P.n, 3))
        t[P.free] = (Htrue @ s[P.free].ravel()).reshape(nf, 3)
        hist.append((s, t, O.tr_dot(t, s)))
        pairs.append((s[P.free].ravel(), t[P.free].ravel()))
    A = O.assemble_A(P).toarray()
    H = np.kron(np.linalg.inv(A), np.eye(3))  # free entries as (vertex, coordinate), row-major
    I = np.eye(3 * nf)
    for s, t in pairs:
        r = 1.0 / (t @ s)
        H = (I - r * np.outer(s, t)) @ H @ (I - r * np.outer(t, s)) + r * np.outer(s, s)
    g = np.zeros((P.n, 3))
    g[P.free] = rng.normal(size=(nf, 3))
    d = O.lbfgs_direction(P, g, hist)
    expect = -(H @ g[P.free].ravel())
    np.testing.assert_allclose(d[P.free].ravel(), expect, rtol=1e-9, atol=1e-12 * np.abs(expect).max())
    assert np.all(d[~np.isin(np.arange(P.n), P.free)] == 0.0)


# ---------------------------------------------------------------- Alg. 2's window, Alg. 1's trial cap

def _iterate_gradients(P, w, iterates):
    y = O.predictor(P, w.q_cur, w.q_prev)
    return y, [O.gradient(P, x, y) for x in iterates]


def test_history_window_keeps_the_newest_m_pairs():
    """Alg. 2 (Sec. 4.2) builds the direction of iteration k from the newest
    min(m, k - 1) accepted pairs (s, t).  With m = 2 over ten iterations the
    window evicts from the fourth iteration on.  Rebuilding every pair from
    the step's accepted iterates and their gradients, and each direction from
    exactly the newest pairs, reproduces every step x_{k+1} - x_k = alpha_k d_k
    the oracle took (alpha_k = 1/2^(trials - 1)).  A window that evicted the
    newest pair, or never evicted, gives other steps: both are checked to
    fail, so the pin is sensitive to the eviction rule."""
    w = W.lattice_workload((3, 3, 3), W.Material(W.NEOHOOKEAN, 1e5, 0.45), seed=5, v_range=0.5)
    P = O.problem_from_workload(w)
    m, iters = 2, 10
    _, st, its = O.solve_step(P, w.q_cur, w.q_prev, iters=iters, m=m, return_iterates=True)
    assert st.resets == 0 and not st.exhausted and len(its) == iters + 1
    y, grads = _iterate_gradients(P, w, its)
    pairs = []
    for k in range(iters):
        s, t = its[k + 1] - its[k], grads[k + 1] - grads[k]
        rho = O.tr_dot(t, s)
        # every pair passes the curvature filter with room to spare, so the
        # window is the plain "newest m" of the accepted pairs
        assert rho > 1e-6 * np.linalg.norm(s) * np.linalg.norm(t)
        pairs.append((s, t, rho))

    def steps_with(window):
        out = []
        for k in range(iters):
            d = O.lbfgs_direction(P, grads[k], window(k))
            alpha = 0.5 ** (st.trials[k] - 1)
            out.append(alpha * d)
        return out

    taken = [its[k + 1] - its[k] for k in range(iters)]
    newest = steps_with(lambda k: pairs[max(0, k - m):k])
    for k in range(iters):
        assert np.linalg.norm(newest[k] - taken[k]) <= 1e-12 * np.linalg.norm(taken[k]), k
    evict_newest = steps_with(lambda k: pairs[:min(k, m - 1)] + pairs[k - 1:k] if k > m else pairs[:k])
    keep_all = steps_with(lambda k: pairs[:k])
    for alt in (evict_newest, keep_all):
        worst = max(np.linalg.norm(alt[k] - taken[k]) / np.linalg.norm(taken[k]) for k in range(m + 1, iters))
        assert worst > 1e-6, worst


def test_line_search_exhaustion_keeps_x_k_and_ends_the_step():
    """Alg. 1 with a cap of ls_max trials (the paper gives none): when every
    trial is rejected the step keeps x_k, reports the exhaustion and runs no
    further iterations.  On the small twisted spline bar the ninth iteration
    rejects alpha = 1 (checked here from Armijo's inequality itself:
    g(x_k + d) > g(x_k) + 0.3 tr(grad^T d)) and accepts alpha = 1/2.  With
    ls_max = 1 the step ends there at x_k; with ls_max = 2 it runs as
    uncapped."""
    w = W.spline_bar_80x40x40(scale=16)
    P = O.problem_from_workload(w)
    _, st_full, its_full = O.solve_step(P, w.q_cur, w.q_prev, iters=10, m=5, return_iterates=True)
    assert max(st_full.trials) == 2
    k0 = st_full.trials.index(2)
    assert k0 >= 5  # the history window is full when the rejection happens
    y, grads = _iterate_gradients(P, w, its_full[:k0 + 1])
    d = (its_full[k0 + 1] - its_full[k0]) / 0.5
    g_k = O.objective(P, its_full[k0], y)
    gd = O.tr_dot(grads[k0], d)
    assert gd < 0
    assert O.objective(P, its_full[k0] + d, y) > g_k + 0.3 * gd
    assert O.objective(P, its_full[k0] + 0.5 * d, y) <= g_k + 0.3 * 0.5 * gd

    x1, st1, its1 = O.solve_step(P, w.q_cur, w.q_prev, iters=10, m=5, ls_max=1, return_iterates=True)
    assert st1.exhausted
    assert st1.trials == [1] * (k0 + 1)
    assert len(its1) == k0 + 1
    np.testing.assert_array_equal(x1, its_full[k0])
    assert st1.g[-1] == pytest.approx(g_k, rel=1e-14)

    x2, st2 = O.solve_step(P, w.q_cur, w.q_prev, iters=10, m=5, ls_max=2)
    assert not st2.exhausted and st2.trials == st_full.trials
    np.testing.assert_array_equal(x2, its_full[-1])


# ---------------------------------------------------------------- several materials in one mesh

def _submesh_problem(w, mat, sel):
    """The same vertices with only the tets `sel`, all of material `mat`."""
    return O.build_problem(w.rest_pos, w.tets[sel], w.clamped, O._material_of(mat), mat.density, w.h, w.gravity)


def test_two_materials_are_the_sum_of_their_parts():
    """Eq. PD's energy and L are sums over elements, each with its own
    material: on a bar of Neo-Hookean and StVK halves (different densities),
    the elastic energy, its gradient, the lumped mass and L equal those of
    the two single-material halves added up (independently built
    problems); with both materials equal the mesh is the one-material mesh."""
    a = W.Material(W.NEOHOOKEAN, 2e5, 0.4, density=900.0)
    b = W.Material(W.STVK, 6e5, 0.35, density=1300.0)
    w = W.two_material_bar((4, 2, 3), a, b, seed=3, v_range=0.2)
    P = O.problem_from_workload(w)
    assert set(np.unique(P.tmat)) == {0, 1} and P.k_tet.min() < P.k_tet.max()
    P0 = _submesh_problem(w, a, w.tet_material == 0)
    P1 = _submesh_problem(w, b, w.tet_material == 1)
    rng = np.random.default_rng(8)
    x = w.q_cur + 3e-3 * rng.normal(size=w.q_cur.shape)
    e = O.elastic_energy_per_tet(P, x)
    assert abs(e.sum() - (O.elastic_energy_per_tet(P0, x).sum() + O.elastic_energy_per_tet(P1, x).sum())) \
        <= 1e-12 * abs(e.sum())
    np.testing.assert_allclose(P.mass, P0.mass + P1.mass, rtol=1e-14)
    y = w.q_cur.copy()
    # the inertia term splits with the mass: g = g_0 + g_1
    g = O.gradient(P, x, y)
    np.testing.assert_allclose(g, O.gradient(P0, x, y) + O.gradient(P1, x, y), rtol=1e-10,
                               atol=1e-12 * np.abs(g).max())
    assert abs(O.objective(P, x, y) - O.objective(P0, x, y) - O.objective(P1, x, y)) <= 1e-12 * O.objective(P, x, y)
    Lsum = (O.laplacian(P0) + O.laplacian(P1)).toarray()
    np.testing.assert_allclose(O.laplacian(P).toarray(), Lsum, rtol=1e-12, atol=1e-12 * np.abs(Lsum).max())
    # both halves of one material: the one-material mesh, bit for bit
    w2 = W.two_material_bar((4, 2, 3), a, a, seed=3, v_range=0.2)
    Pa, Pone = O.problem_from_workload(w2), _submesh_problem(w2, a, slice(None))
    np.testing.assert_array_equal(O.gradient(Pa, x, y), O.gradient(Pone, x, y))
    assert O.objective(Pa, x, y) == O.objective(Pone, x, y)


def test_two_materials_gradient_matches_central_differences():
    a = W.Material(W.NEOHOOKEAN, 2e5, 0.4, density=900.0)
    b = W.Material(W.COROTATED, 6e5, 0.35, density=1300.0)
    w = W.two_material_bar((3, 2, 2), a, b, seed=4)
    P = O.problem_from_workload(w)
    rng = np.random.default_rng(2)
    x = w.q_cur + 4e-3 * rng.normal(size=w.q_cur.shape)
    y = w.q_cur + 1e-3 * rng.normal(size=w.q_cur.shape)
    g = O.gradient(P, x, y)
    eps = 1e-6
    for v in P.free[::3]:
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, c] += eps
            xm[v, c] -= eps
            fd = (O.objective(P, xp, y) - O.objective(P, xm, y)) / (2 * eps)
            assert abs(fd - g[v, c]) <= 1e-6 * max(1.0, abs(g[v, c])), (v, c, fd, g[v, c])


def test_chebyshev_rho_estimate_matches_the_spectral_radius():
    """The rho estimate from a projective-dynamics run's objective values
    (paper_1604_07378_gb300/chebyshev.py) against the spectral radius of the
    iteration's linearisation at the minimiser, I - A0^{-1} H with H the
    (finite-difference) Hessian of g at x*, by a dense eigensolve on a tiny
    mesh."""
    from paper_1604_07378_gb300 import chebyshev
    w, P = _problem((2, 2, 3), kind=W.STVK, v=0.6, seed=9)
    x_star, _ = O.newton_minimise(P, w.q_cur, w.q_prev)
    y = O.predictor(P, w.q_cur, w.q_prev)
    free, nf = P.free, P.free.size
    eps = 1e-7
    H = np.zeros((3 * nf, 3 * nf))
    for j in range(3 * nf):
        vj, cj = divmod(j, 3)
        xp, xm = x_star.copy(), x_star.copy()
        xp[free[vj], cj] += eps
        xm[free[vj], cj] -= eps
        H[:, j] = (O.gradient(P, xp, y)[free].ravel() - O.gradient(P, xm, y)[free].ravel()) / (2 * eps)
    A = np.kron(O.assemble_A(P).toarray(), np.eye(3))
    rho_exact = float(np.max(np.abs(np.linalg.eigvals(np.eye(3 * nf) - np.linalg.solve(A, 0.5 * (H + H.T))))))
    assert 0.3 < rho_exact < 1.0
    # the slowest mode dominates once the faster ones have died out
    _, st = O.solve_step(P, w.q_cur, w.q_prev, iters=150, m=0)
    rho = chebyshev.estimate_rho([st.g0] + st.g)
    assert abs(rho - rho_exact) <= 0.01 * rho_exact, (rho, rho_exact)
