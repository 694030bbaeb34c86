"""CPU FP64 oracle for the quasi-Newton / L-BFGS implicit-Euler solver.

TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously correct restatement
of Liu, Bouaziz & Kavan, "Towards Real-time Simulation of Hyperelastic
Materials" (2016/2017), in float64 numpy/scipy.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the library never
does, and it shares no code with the CUDA path.

Where the paper is silent the oracle takes these readings (each one is also
taken by the CUDA path, written separately):
  * lumped mass m_v = density * sum of incident tet volumes / 4;
  * projective-dynamics element energy read as (w/2)||G x - p||^2, so that
    L = sum_t w_t G_t^T G_t with w_t = V_t k_t (Eq. PDtotalEnergy, PDmatrixForm);
  * stiffness k = continuous least-squares slope of a'(s) + 2b'(s) + c'(s)
    over [x_start, x_end] = [0.5, 1.5] (Eq. stiffness), by Gauss-Legendre
    quadrature split at the material's breakpoints (spline knots, J0);
  * Neo-Hookean in Valanis-Landel form a = mu/2 (x^2 - 1), b = 0,
    c(J) = -mu ln J + lam/2 ln^2 J, with c replaced by its second-order Taylor
    polynomial at J0 = 0.05 for J < J0 (finite for inverted tets);
  * signed SVD: U, V in SO(3), s1 >= s2 >= |s3|, s3 < 0 iff det F < 0;
  * clamped vertices keep prescribed positions; y there equals that position;
  * L-BFGS history is reset at the start of every time step; a pair is kept
    only if rho = tr(t^T s) > 1e-12 ||s|| ||t||; if tr(grad^T d) >= 0 the
    history is dropped and d = -A0^{-1} grad;
  * the backtracking line search gives up after ls_max trials, keeping x_k and
    ending the step's iterations;
  * a mesh may give each tet its own material (the energy of Eq. PD is a sum
    over elements): a tet's energy density, its mass share (density * V / 4)
    and its weight V k in L use its own material, k fitted per material;
  * the anisotropic fibre term kappa/2 (|F d| - 1)^2 of Sec. 4.4 is added to
    the base material's energy density; A0 keeps the base material's
    stiffness fit (Eq. stiffness is defined for Valanis-Landel energies only);
  * the iterative alternative to A0^{-1} (Sec. 8's comparison): Jacobi-
    preconditioned CG from zero with a fixed number of iterations, the three
    coordinate columns treated as one vector (one alpha, one beta);
  * Alg. 3 (the Chebyshev direction) reads x_0 := x_1 (its first S
    directions have omega = 1, where x_{k-1} cancels) and keeps no history;
  * collisions (Sec. 4.3) against analytic colliders (a plane with its
    normal, a sphere the body stays outside of, or a torus -- the paper's
    examples are a ground plane and a torus): at the start of every
    iteration, before the gradient at x_k, each free vertex that penetrates a
    collider (signed distance < 0) and does not move away from it (its
    displacement over the step, x_k - q_l, has a non-positive normal
    component) gets the term w_v ((x - t)^T n)^2 with t its projection on the
    surface and n the surface normal there, both frozen for the iteration;
    w_v = contact_scale * m_v / h^2 (the paper prints no weight).  The terms
    enter the objective and its gradient but not A0.

Parity pins: see tests/test_oracle_pins.py (finite differences, rest state,
invariances, invariant-form materials, closed-form stiffness, SPD and residual
of A0, secant condition, m = 0 reduction, the projective-dynamics identity,
centre-of-mass motion, convergence to a Newton minimiser).  One branch has
no pin: the non-descent reset of solve_step (parity unpinned).  With every
kept pair's rho > 0 the L-BFGS matrix is positive definite, so the branch is
a safeguard against rounding that no input tried has reached.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

NEOHOOKEAN, STVK, SPLINE_VL, COROTATED, POLY4 = 0, 1, 2, 3, 4
J0_NEOHOOKEAN = 0.05


# ----------------------------------------------------------------------------
# Materials in Valanis-Landel form (Eq. valanis-landel):
#   Psi(s1,s2,s3) = sum_i a(s_i) + sum_{i<j} b(s_i s_j) + c(s1 s2 s3)
# Each material gives a, a', b, b', c, c' as vectorised numpy functions.
# ----------------------------------------------------------------------------

class VLMaterial:
    # anisotropic fibre term kappa/2 (|F d| - 1)^2 (Sec. 4.4) on top of the
    # stretch energy; kappa = 0: none.  It is not Valanis-Landel and does not
    # enter the stiffness fit (A0 keeps the base material's).
    kappa = 0.0
    fiber = (0.0, 0.0, 0.0)

    def breakpoints(self): return ()
    def a(self, x): return np.zeros_like(x)
    def da(self, x): return np.zeros_like(x)
    def b(self, y): return np.zeros_like(y)
    def db(self, y): return np.zeros_like(y)
    def c(self, J): return np.zeros_like(J)
    def dc(self, J): return np.zeros_like(J)


class NeoHookean(VLMaterial):
    """Psi = mu/2 (I1 - 3) - mu ln J + lam/2 ln^2 J in principal stretches."""

    def __init__(self, mu, lam, J0=J0_NEOHOOKEAN):
        self.mu, self.lam, self.J0 = mu, lam, J0

    def breakpoints(self): return (self.J0,)

    def a(self, x): return 0.5 * self.mu * (x * x - 1.0)
    def da(self, x): return self.mu * x

    def _c_exact(self, J):
        lj = np.log(J)
        return -self.mu * lj + 0.5 * self.lam * lj * lj

    def _dc_exact(self, J):
        return (-self.mu + self.lam * np.log(J)) / J

    def _ddc_exact(self, J):
        return (self.mu + self.lam - self.lam * np.log(J)) / (J * J)

    def c(self, J):
        J = np.asarray(J, dtype=np.float64)
        J0 = self.J0
        Jc = np.where(J >= J0, J, J0)
        exact = self._c_exact(Jc)
        dJ = J - J0
        taylor = (self._c_exact(J0) + self._dc_exact(J0) * dJ
                  + 0.5 * self._ddc_exact(J0) * dJ * dJ)
        return np.where(J >= J0, exact, taylor)

    def dc(self, J):
        J = np.asarray(J, dtype=np.float64)
        J0 = self.J0
        Jc = np.where(J >= J0, J, J0)
        exact = self._dc_exact(Jc)
        taylor = self._dc_exact(J0) + self._ddc_exact(J0) * (J - J0)
        return np.where(J >= J0, exact, taylor)


class StVK(VLMaterial):
    """Psi = mu ||E||^2 + lam/2 tr^2 E with E = (F^T F - I)/2, in VL form."""

    def __init__(self, mu, lam):
        self.mu, self.lam = mu, lam

    def a(self, x):
        e = x * x - 1.0
        return (0.25 * self.mu + 0.125 * self.lam) * e * e - 0.5 * self.lam * e

    def da(self, x):
        e = x * x - 1.0
        return (self.mu + 0.5 * self.lam) * e * x - self.lam * x

    def b(self, y): return 0.25 * self.lam * (y * y - 1.0)
    def db(self, y): return 0.5 * self.lam * y


class Corotated(VLMaterial):
    """a = mu (x-1)^2, c = lam/2 (J-1)^2 (lam = 0 gives as-rigid-as-possible)."""

    def __init__(self, mu, lam):
        self.mu, self.lam = mu, lam

    def a(self, x): return self.mu * (x - 1.0) ** 2
    def da(self, x): return 2.0 * self.mu * (x - 1.0)
    def c(self, J): return 0.5 * self.lam * (J - 1.0) ** 2
    def dc(self, J): return self.lam * (J - 1.0)


class Poly4(VLMaterial):
    """The paper's polynomial material a(x) = mu (x-1)^4, b = c = 0."""

    def __init__(self, mu):
        self.mu = mu

    def a(self, x): return self.mu * (x - 1.0) ** 4
    def da(self, x): return 4.0 * self.mu * (x - 1.0) ** 3


class HermiteSpline:
    """C1 piecewise cubic Hermite interpolant through (knot, value, slope),
    extended outside the knots by the quadratic Taylor polynomial of the
    end segment at the end knot."""

    def __init__(self, pts):
        pts = np.asarray(pts, dtype=np.float64)
        self.x, self.v, self.s = pts[:, 0], pts[:, 1], pts[:, 2]

    def _segment(self, t):
        i = np.clip(np.searchsorted(self.x, t, side="right") - 1, 0, self.x.size - 2)
        return i

    def _eval(self, t, i):
        x0, x1 = self.x[i], self.x[i + 1]
        hh = x1 - x0
        u = (t - x0) / hh
        h00 = 2 * u**3 - 3 * u**2 + 1
        h10 = u**3 - 2 * u**2 + u
        h01 = -2 * u**3 + 3 * u**2
        h11 = u**3 - u**2
        val = h00 * self.v[i] + h10 * hh * self.s[i] + h01 * self.v[i + 1] + h11 * hh * self.s[i + 1]
        d00 = (6 * u**2 - 6 * u) / hh
        d10 = 3 * u**2 - 4 * u + 1
        d01 = (-6 * u**2 + 6 * u) / hh
        d11 = 3 * u**2 - 2 * u
        der = d00 * self.v[i] + d10 * self.s[i] + d01 * self.v[i + 1] + d11 * self.s[i + 1]
        e00 = (12 * u - 6) / hh**2
        e10 = (6 * u - 4) / hh
        e01 = (-12 * u + 6) / hh**2
        e11 = (6 * u - 2) / hh
        sec = e00 * self.v[i] + e10 * self.s[i] + e01 * self.v[i + 1] + e11 * self.s[i + 1]
        return val, der, sec

    def value_and_slope(self, t):
        t = np.asarray(t, dtype=np.float64)
        lo, hi = self.x[0], self.x[-1]
        tc = np.clip(t, lo, hi)
        i = self._segment(tc)
        val, der, sec = self._eval(tc, i)
        dt = t - tc            # zero inside the knots
        return val + der * dt + 0.5 * sec * dt * dt, der + sec * dt

    def __call__(self, t): return self.value_and_slope(t)[0]
    def deriv(self, t): return self.value_and_slope(t)[1]


class SplineVL(VLMaterial):
    """Spline-based Valanis-Landel material: a, b, c are Hermite splines."""

    def __init__(self, control):
        control = np.asarray(control, dtype=np.float64)
        self.sa, self.sb, self.sc = (HermiteSpline(control[f]) for f in range(3))

    def breakpoints(self):
        return tuple(self.sa.x) + tuple(self.sb.x) + tuple(self.sc.x)

    def a(self, x): return self.sa(x)
    def da(self, x): return self.sa.deriv(x)
    def b(self, y): return self.sb(y)
    def db(self, y): return self.sb.deriv(y)
    def c(self, J): return self.sc(J)
    def dc(self, J): return self.sc.deriv(J)


def lame(E, nu):
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def make_material(kind, E, nu, spline=None) -> VLMaterial:
    mu, lam = lame(E, nu)
    if kind == NEOHOOKEAN:
        return NeoHookean(mu, lam)
    if kind == STVK:
        return StVK(mu, lam)
    if kind == SPLINE_VL:
        return SplineVL(spline)
    if kind == COROTATED:
        return Corotated(mu, lam)
    if kind == POLY4:
        return Poly4(mu)
    raise ValueError(f"unknown material kind {kind}")


def psi(mat: VLMaterial, s):
    """Energy density from principal stretches s (..., 3), Eq. valanis-landel."""
    s1, s2, s3 = s[..., 0], s[..., 1], s[..., 2]
    return (mat.a(s1) + mat.a(s2) + mat.a(s3)
            + mat.b(s1 * s2) + mat.b(s2 * s3) + mat.b(s1 * s3)
            + mat.c(s1 * s2 * s3))


def dpsi(mat: VLMaterial, s):
    """d Psi / d s_i (..., 3) by the chain rule on Eq. valanis-landel."""
    s1, s2, s3 = s[..., 0], s[..., 1], s[..., 2]
    J = s1 * s2 * s3
    dcJ = mat.dc(J)
    g1 = mat.da(s1) + mat.db(s1 * s2) * s2 + mat.db(s1 * s3) * s3 + dcJ * s2 * s3
    g2 = mat.da(s2) + mat.db(s1 * s2) * s1 + mat.db(s2 * s3) * s3 + dcJ * s1 * s3
    g3 = mat.da(s3) + mat.db(s2 * s3) * s2 + mat.db(s1 * s3) * s1 + dcJ * s1 * s2
    return np.stack([g1, g2, g3], axis=-1)


def stiffness_k(mat: VLMaterial, x_start=0.5, x_end=1.5, npts=64):
    """Eq. stiffness: slope of the least-squares line through
    f(s) = a'(s) + 2 b'(s) + c'(s) on [x_start, x_end] (continuous fit),
    k = int (s - sbar) f ds / int (s - sbar)^2 ds.  The integral is split at
    the material's breakpoints (spline knots, the Neo-Hookean J0) so that each
    piece is smooth; Gauss-Legendre with npts nodes per piece."""
    t, w = np.polynomial.legendre.leggauss(npts)
    mid = 0.5 * (x_end + x_start)
    cuts = sorted({x_start, x_end} | {float(b) for b in mat.breakpoints() if x_start < b < x_end})
    num = 0.0
    for a, b in zip(cuts[:-1], cuts[1:]):
        half = 0.5 * (b - a)
        s = 0.5 * (a + b) + half * t
        f = mat.da(s) + 2.0 * mat.db(s) + mat.dc(s)
        num += half * np.sum(w * (s - mid) * f)
    den = (x_end - x_start) ** 3 / 12.0
    return num / den


# ----------------------------------------------------------------------------
# Signed SVD (invertible-element convention) using the library SVD as a step.
# ----------------------------------------------------------------------------

def signed_svd(F):
    """F (..., 3, 3) -> U, s, V with F = U diag(s) V^T, U, V in SO(3),
    s1 >= s2 >= |s3| and s3 < 0 exactly when det F < 0."""
    U, s, Vt = np.linalg.svd(F)
    V = np.swapaxes(Vt, -1, -2).copy()
    U = U.copy()
    s = s.copy()
    du = np.linalg.det(U) < 0
    U[du, :, 2] *= -1.0
    s[du, 2] *= -1.0
    dv = np.linalg.det(V) < 0
    V[dv, :, 2] *= -1.0
    s[dv, 2] *= -1.0
    return U, s, V


# ----------------------------------------------------------------------------
# The simulated object: rest data, mass, stiffness weights, A0 = M/h^2 + L.
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    X: np.ndarray            # rest positions (n, 3)
    tets: np.ndarray         # (T, 4)
    clamped: np.ndarray      # (n,) bool
    mat: VLMaterial
    density: float
    h: float
    gravity: np.ndarray
    Dm_inv: np.ndarray = None
    vol: np.ndarray = None
    mass: np.ndarray = None
    k: float = None
    free: np.ndarray = None
    A: sp.csc_matrix = None
    _solver: object = None
    colliders: tuple = ()        # ("plane", point, normal), ("sphere", centre, radius) or
                                 # ("torus", centre, axis, ring radius, tube radius)
    contact_scale: float = 100.0
    mats: tuple = ()             # the materials of a mesh with several (mats[0] is `mat`)
    tmat: np.ndarray = None      # (T,) index of each tet's material in mats
    k_tet: np.ndarray = None     # (T,) stiffness k of each tet's material

    @property
    def n(self): return self.X.shape[0]


def build_problem(X, tets, clamped, mat, density, h, gravity,
                  x_start=0.5, x_end=1.5, colliders=(), contact_scale=100.0, tet_material=None) -> Problem:
    """mat and density: one material and its density, or (with tet_material,
    each tet's index into them) sequences of them."""
    X = np.asarray(X, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    mats = tuple(mat) if isinstance(mat, (list, tuple)) else (mat,)
    dens = np.atleast_1d(np.asarray(density, dtype=np.float64))
    tmat = np.zeros(tets.shape[0], dtype=np.int64) if tet_material is None else np.asarray(tet_material, np.int64)
    P = Problem(X=X, tets=tets, clamped=np.asarray(clamped).astype(bool), mat=mats[0],
                density=float(dens[0]), h=float(h), gravity=np.asarray(gravity, dtype=np.float64))
    P.mats, P.tmat = mats, tmat
    # rest shape matrices Dm = [X1-X0, X2-X0, X3-X0] (columns), volume det(Dm)/6
    Dm = np.stack([X[tets[:, 1]] - X[tets[:, 0]], X[tets[:, 2]] - X[tets[:, 0]],
                   X[tets[:, 3]] - X[tets[:, 0]]], axis=-1)
    det = np.linalg.det(Dm)
    if np.any(det <= 0):
        raise ValueError("degenerate or negatively oriented rest tet")
    P.Dm_inv = np.linalg.inv(Dm)
    P.vol = det / 6.0
    # lumped mass: a quarter of each incident tet's mass
    mass = np.zeros(P.n)
    for c in range(4):
        np.add.at(mass, tets[:, c], 0.25 * dens[tmat] * P.vol)
    P.mass = mass
    ks = np.array([stiffness_k(m, x_start, x_end) for m in mats])
    P.k = float(ks[0])
    P.k_tet = ks[tmat]
    P.free = np.flatnonzero(~P.clamped)
    P.A = assemble_A(P)
    P.colliders = tuple(colliders)
    P.contact_scale = float(contact_scale)
    return P


def laplacian(P: Problem, weights=None):
    """L = sum_t w_t G_t^T G_t (n x n), w_t = V_t k_t (Eq. PDmatrixForm), k_t
    the stiffness of tet t's material.
    G_t maps positions to Dm^{-T} [x1-x0; x2-x0; x3-x0]."""
    w = P.vol * P.k_tet if weights is None else weights
    B = np.array([[-1.0, 1.0, 0.0, 0.0], [-1.0, 0.0, 1.0, 0.0], [-1.0, 0.0, 0.0, 1.0]])
    # G_t = Dm^{-T} B  (3 x 4 on the tet's vertices)
    G = np.einsum("tji,jk->tik", P.Dm_inv, B)
    K = w[:, None, None] * np.einsum("tia,tib->tab", G, G)
    rows = np.repeat(P.tets, 4, axis=1).ravel()
    cols = np.tile(P.tets, (1, 4)).ravel()
    return sp.csr_matrix((K.ravel(), (rows, cols)), shape=(P.n, P.n))


def assemble_A(P: Problem):
    """A0 = M/h^2 + L restricted to the free vertices (Eq. PDsolution)."""
    L = laplacian(P)
    A = L + sp.diags(P.mass / P.h**2)
    A = A.tocsr()[P.free][:, P.free]
    return A.tocsc()


def solve_A(P: Problem, q):
    """r = A0^{-1} q on the free vertices, 3 right-hand sides (x, y, z)."""
    if P._solver is None:
        P._solver = spla.splu(P.A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                              options=dict(SymmetricMode=True))
    out = np.zeros_like(q)
    out[P.free] = P._solver.solve(np.ascontiguousarray(q[P.free]))
    return out


def jacobi_diagonal(P: Problem):
    """diag(A0) on the free vertices (the Jacobi preconditioner)."""
    return np.asarray(P.A.diagonal()).ravel()


def solve_A_pcg(P: Problem, q, iters):
    """An approximation of A0^{-1} q by `iters` iterations of Jacobi-
    preconditioned conjugate gradients from zero (the paper's comparison
    with iterative solvers, Sec. 8): the three right-hand sides form one
    vector (inner products tr(a^T b)), so every iteration has one step
    length alpha and one beta.  Stops early only if the residual vanishes."""
    out = np.zeros_like(q)
    b = np.ascontiguousarray(q[P.free])
    dinv = 1.0 / jacobi_diagonal(P)
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv[:, None] * r
    p = z.copy()
    rz = tr_dot(r, z)
    for _ in range(iters):
        if rz == 0.0:
            break
        Ap = P.A @ p
        alpha = rz / tr_dot(p, Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        z = dinv[:, None] * r
        rz_new = tr_dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    out[P.free] = x
    return out


# ----------------------------------------------------------------------------
# Objective g(x) of Eq. PD and its gradient.
# ----------------------------------------------------------------------------

def deformation_gradients(P: Problem, x):
    Ds = np.stack([x[P.tets[:, 1]] - x[P.tets[:, 0]], x[P.tets[:, 2]] - x[P.tets[:, 0]],
                   x[P.tets[:, 3]] - x[P.tets[:, 0]]], axis=-1)
    return Ds @ P.Dm_inv


def fiber_stretch(mat: VLMaterial, F):
    """F d and |F d| for the material's fibre direction d (Sec. 4.4)."""
    d = np.asarray(mat.fiber, dtype=np.float64)
    Fd = F @ d
    return Fd, np.linalg.norm(Fd, axis=1)


def material_groups(P: Problem):
    """(material, boolean mask of its tets) for every material of the mesh."""
    if len(P.mats) <= 1:
        return [(P.mat, slice(None))]
    return [(m, P.tmat == i) for i, m in enumerate(P.mats)]


def elastic_energy_per_tet(P: Problem, x):
    """V (Psi(s) + kappa/2 (|F d| - 1)^2): the Valanis-Landel energy of the
    stretches plus the anisotropic fibre term of Sec. 4.4 (kappa = 0: none),
    each tet with its own material."""
    F = deformation_gradients(P, x)
    _, s, _ = signed_svd(F)
    e = np.zeros(P.tets.shape[0])
    for mat, sel in material_groups(P):
        e[sel] = psi(mat, s[sel])
        if mat.kappa:
            _, nrm = fiber_stretch(mat, F[sel])
            e[sel] = e[sel] + 0.5 * mat.kappa * (nrm - 1.0) ** 2
    return P.vol * e


def elastic_corner_gradients(P: Problem, x):
    """d(V Psi)/dx for the 4 corners of every tet, (T, 4, 3).
    P = U diag(dPsi/ds) V^T; corners 1..3 are the columns of V P Dm^{-T},
    corner 0 is minus their sum."""
    F = deformation_gradients(P, x)
    U, s, V = signed_svd(F)
    tau = np.zeros_like(s)
    for mat, sel in material_groups(P):
        tau[sel] = dpsi(mat, s[sel])
    Pk = U @ (tau[:, :, None] * np.swapaxes(V, -1, -2))
    for mat, sel in material_groups(P):
        if mat.kappa:
            # d/dF kappa/2 (|F d| - 1)^2 = kappa (|F d| - 1) (F d / |F d|) d^T
            d = np.asarray(mat.fiber, dtype=np.float64)
            Fd, nrm = fiber_stretch(mat, F[sel])
            Pk[sel] = Pk[sel] + (mat.kappa * (nrm - 1.0) / nrm)[:, None, None] * (Fd[:, :, None] * d[None, None, :])
    H = P.vol[:, None, None] * (Pk @ np.swapaxes(P.Dm_inv, -1, -2))
    out = np.zeros((P.tets.shape[0], 4, 3))
    out[:, 1:, :] = np.swapaxes(H, -1, -2)
    out[:, 0, :] = -out[:, 1:, :].sum(axis=1)
    return out


# ----------------------------------------------------------------------------
# Collision terms (Sec. 4.3).
# ----------------------------------------------------------------------------

@dataclass
class Contacts:
    """Active collision terms of one iteration: vertex ids, surface points t,
    unit normals n and weights w (term w ((x_v - t)^T n)^2)."""
    idx: np.ndarray
    t: np.ndarray
    n: np.ndarray
    w: np.ndarray


def contact_terms(P: Problem, x, q_ref):
    """The terms active at the iterate x: free vertices with negative signed
    distance to a collider whose displacement x - q_ref does not point away
    from it (q_ref: the position at the start of the time step)."""
    idx, ts, ns, ws = [], [], [], []
    free = np.zeros(P.n, dtype=bool)
    free[P.free] = True
    for col in P.colliders:
        if col[0] == "plane":
            p, nrm = np.asarray(col[1], float), np.asarray(col[2], float)
            nrm = nrm / np.linalg.norm(nrm)
            phi = (x - p) @ nrm
            n = np.broadcast_to(nrm, x.shape)
        elif col[0] == "sphere":
            c, r = np.asarray(col[1], float), float(col[2])
            rel = x - c
            dist = np.linalg.norm(rel, axis=1)
            phi = np.where(dist > 0.0, dist - r, np.inf)  # at the centre: no normal, no term
            n = rel / np.maximum(dist, 1e-300)[:, None]
        elif col[0] == "torus":
            # ring of radius R about the axis a through c, tube radius r: the
            # nearest surface point lies on the segment from x to the nearest
            # point of the ring circle, at distance r from that point
            c, a = np.asarray(col[1], float), np.asarray(col[2], float)
            R, r = float(col[3]), float(col[4])
            a = a / np.linalg.norm(a)
            rel = x - c
            radial = rel - np.outer(rel @ a, a)
            rho = np.linalg.norm(radial, axis=1)
            v = rel - (R / np.maximum(rho, 1e-300))[:, None] * radial
            dist = np.linalg.norm(v, axis=1)
            # on the axis or on the ring circle: no unique normal, no term
            phi = np.where((rho > 0.0) & (dist > 0.0), dist - r, np.inf)
            n = v / np.maximum(dist, 1e-300)[:, None]
        else:
            raise ValueError(f"unknown collider {col[0]!r}")
        vn = np.sum((x - q_ref) * n, axis=1)
        act = np.flatnonzero(free & (phi < 0.0) & (vn <= 0.0))
        idx.append(act)
        ts.append(x[act] - phi[act, None] * n[act])
        ns.append(n[act])
        ws.append(P.contact_scale * P.mass[act] / P.h**2)
    if not idx:
        z = np.zeros(0, dtype=np.int64)
        return Contacts(z, np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    return Contacts(np.concatenate(idx), np.concatenate(ts), np.concatenate(ns), np.concatenate(ws))


def contact_energy(C: Contacts, x):
    if C is None or C.idx.size == 0:
        return 0.0
    gap = np.sum((x[C.idx] - C.t) * C.n, axis=1)
    return float(np.sum(C.w * gap * gap))


def contact_gradient(C: Contacts, x, grad):
    if C is None or C.idx.size == 0:
        return grad
    gap = np.sum((x[C.idx] - C.t) * C.n, axis=1)
    np.add.at(grad, C.idx, (2.0 * C.w * gap)[:, None] * C.n)
    return grad


def objective(P: Problem, x, y, contacts: Contacts = None):
    """g(x) = 1/(2h^2) tr((x-y)^T M (x-y)) + E(x), Eq. PD (free vertices),
    plus the active collision terms (Sec. 4.3) if any."""
    dx = (x - y)[P.free]
    inertia = 0.5 / P.h**2 * np.sum(P.mass[P.free, None] * dx * dx)
    return inertia + np.sum(elastic_energy_per_tet(P, x)) + contact_energy(contacts, x)


def gradient(P: Problem, x, y, contacts: Contacts = None):
    """grad g = M (x - y)/h^2 + grad E (+ the collision terms), zero on
    clamped vertices."""
    cg = elastic_corner_gradients(P, x)
    grad = np.zeros_like(x)
    for c in range(4):
        np.add.at(grad, P.tets[:, c], cg[:, c, :])
    grad += P.mass[:, None] * (x - y) / P.h**2
    contact_gradient(contacts, x, grad)
    grad[P.clamped] = 0.0
    return grad


def predictor(P: Problem, q_cur, q_prev):
    """y = 2 q_l - q_{l-1} + h^2 M^{-1} f_ext (gravity: f_ext = m g), Eq. PD;
    clamped vertices are held at q_l."""
    y = 2.0 * q_cur - q_prev + P.h**2 * P.gravity[None, :]
    y[P.clamped] = q_cur[P.clamped]
    return y


# ----------------------------------------------------------------------------
# Alg. 2 (L-BFGS two-loop recursion with A0 = M/h^2 + L) and Alg. 1.
# ----------------------------------------------------------------------------

def tr_dot(a, b):
    return float(np.sum(a * b))


def lbfgs_direction(P: Problem, grad, history, pcg_iters=0):
    """Alg. 2: q := -grad; newest-to-oldest first loop; r := A0^{-1} q;
    oldest-to-newest second loop; d := r.  history is oldest-first [(s, t, rho)].
    pcg_iters > 0 replaces A0^{-1} q by that many Jacobi-PCG iterations."""
    q = -grad
    zeta = [0.0] * len(history)
    for i in range(len(history) - 1, -1, -1):
        s, t, rho = history[i]
        zeta[i] = tr_dot(s, q) / rho
        q = q - zeta[i] * t
    r = solve_A_pcg(P, q, pcg_iters) if pcg_iters > 0 else solve_A(P, q)
    for i in range(len(history)):
        s, t, rho = history[i]
        eta = tr_dot(t, r) / rho
        r = r + s * (zeta[i] - eta)
    return r


@dataclass
class StepStats:
    trials: list = field(default_factory=list)     # line-search trials per iteration
    g: list = field(default_factory=list)          # g(x_k) after each iteration
    g0: float = 0.0                                # g(x_1)
    exhausted: bool = False
    resets: int = 0                                # non-descent history resets


def chebyshev_omega(k, S, rho, omega_k):
    """omega_{k+1} of Alg. 3: 1 for k < S, 2/(2 - rho^2) at k = S,
    4/(4 - rho^2 omega_k) after."""
    if k < S:
        return 1.0
    if k == S:
        return 2.0 / (2.0 - rho * rho)
    return 4.0 / (4.0 - rho * rho * omega_k)


def solve_step(P: Problem, q_cur, q_prev, iters=10, m=5, gamma=0.3, backtrack=0.5,
               ls_max=30, return_iterates=False, pcg_iters=0, chebyshev=None):
    """One implicit-Euler step by Alg. 1 with the direction of Alg. 2
    (pcg_iters > 0: A0^{-1} by that many Jacobi-PCG iterations).  With
    chebyshev = (S, rho) the direction is Alg. 3's instead (no history):
    q = -A0^{-1} grad, x_hat = x_k + q, d = omega (x_hat - x_{k-1}) + x_{k-1} - x_k
    (x_0 read as x_1: the first S directions have omega = 1).
    Returns (x_{iters+1}, stats[, iterates])."""
    y = predictor(P, q_cur, q_prev)
    x = y.copy()                                   # x_1 := y
    col = contact_terms(P, x, q_cur) if P.colliders else None
    gx = objective(P, x, y, col)
    grad = gradient(P, x, y, col)
    st = StepStats(g0=gx)
    history = []
    iterates = [x.copy()]
    x_prev, omega = x.copy(), 1.0
    for it in range(iters):
        if P.colliders and it > 0:
            # the collision terms are updated at the start of the iteration,
            # before the gradient at x_k (Sec. 4.3); g(x_k) is re-evaluated with them
            gx = objective(P, x, y, col)
        if chebyshev is not None:
            S_c, rho_c = chebyshev
            omega = chebyshev_omega(it + 1, S_c, rho_c, omega)
            q = lbfgs_direction(P, grad, [], pcg_iters)
            d = omega * ((x + q) - x_prev) + x_prev - x
        else:
            d = lbfgs_direction(P, grad, history, pcg_iters)
        gd = tr_dot(grad, d)
        if gd >= 0.0 and history:
            history = []
            st.resets += 1
            d = lbfgs_direction(P, grad, history, pcg_iters)
            gd = tr_dot(grad, d)
        alpha = 1.0 / backtrack
        accepted = False
        for trial in range(ls_max):
            alpha *= backtrack
            x_new = x + alpha * d
            g_new = objective(P, x_new, y, col)
            if g_new <= gx + gamma * alpha * gd:
                accepted = True
                break
        st.trials.append(trial + 1)
        if not accepted:
            st.exhausted = True
            st.g.append(gx)
            break
        if P.colliders:
            col = contact_terms(P, x_new, q_cur)
        grad_new = gradient(P, x_new, y, col)
        x_prev = x
        s = x_new - x
        t = grad_new - grad
        rho = tr_dot(t, s)
        if chebyshev is None and rho > 1e-12 * np.linalg.norm(s) * np.linalg.norm(t):
            history.append((s, t, rho))
            if len(history) > m:
                history.pop(0)
        x, gx, grad = x_new, g_new, grad_new
        st.g.append(gx)
        iterates.append(x.copy())
    if return_iterates:
        return x, st, iterates
    return x, st


def relative_error(g_k, g_0, g_star):
    """Eq. RelativeError: (g(x_k) - g(x*)) / (g(x_0) - g(x*))."""
    return (g_k - g_star) / (g_0 - g_star)


# ----------------------------------------------------------------------------
# Dense Newton minimiser for tiny meshes (used only to pin the converged step).
# ----------------------------------------------------------------------------

def newton_minimise(P: Problem, q_cur, q_prev, tol=1e-11, max_iter=100, fd_eps=1e-7):
    """Minimise g of Eq. PD with Newton's method; the Hessian is a central
    finite difference of the analytic gradient, projected to its positive
    part per eigenvalue, with backtracking.  Tiny meshes only."""
    y = predictor(P, q_cur, q_prev)
    x = y.copy()
    free = P.free
    nf = free.size
    for _ in range(max_iter):
        grad = gradient(P, x, y)
        gfree = grad[free].ravel()
        if np.linalg.norm(gfree) < tol * max(1.0, np.linalg.norm(P.mass)):
            break
        H = np.zeros((3 * nf, 3 * nf))
        for j in range(3 * nf):
            vj, cj = divmod(j, 3)
            xp = x.copy(); xp[free[vj], cj] += fd_eps
            xm = x.copy(); xm[free[vj], cj] -= fd_eps
            H[:, j] = (gradient(P, xp, y)[free].ravel() - gradient(P, xm, y)[free].ravel()) / (2 * fd_eps)
        H = 0.5 * (H + H.T)
        w, Q = np.linalg.eigh(H)
        w = np.maximum(w, 1e-8 * np.max(np.abs(w)))
        step = -(Q @ ((Q.T @ gfree) / w))
        d = np.zeros_like(x)
        d[free] = step.reshape(nf, 3)
        gx = objective(P, x, y)
        gd = tr_dot(grad, d)
        alpha = 1.0
        while objective(P, x + alpha * d, y) > gx + 1e-4 * alpha * gd and alpha > 1e-12:
            alpha *= 0.5
        x = x + alpha * d
    return x, objective(P, x, y)


# ----------------------------------------------------------------------------
# Convenience: build from a workload-like object.
# ----------------------------------------------------------------------------

def _material_of(m):
    mat = make_material(m.kind, m.E, m.nu, m.spline)
    kappa = float(getattr(m, "kappa", 0.0))
    if kappa:
        d = np.asarray(m.fiber, dtype=np.float64)
        mat.fiber, mat.kappa = d / np.linalg.norm(d), kappa
    return mat


def problem_from_workload(w, x_start=0.5, x_end=1.5) -> Problem:
    cols = tuple(c.as_tuple() for c in getattr(w, "colliders", ()))
    extra = tuple(getattr(w, "extra_materials", ()))
    ms = (w.material,) + extra
    mats = [_material_of(m) for m in ms]
    tmat = getattr(w, "tet_material", None) if extra else None
    return build_problem(w.rest_pos, w.tets, w.clamped, mats if extra else mats[0],
                         [m.density for m in ms] if extra else w.material.density, w.h, w.gravity,
                         x_start, x_end, colliders=cols, contact_scale=getattr(w, "contact_scale", 100.0),
                         tet_material=tmat)
