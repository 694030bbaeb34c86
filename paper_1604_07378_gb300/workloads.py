"""Seeded synthetic inputs: tetrahedral lattices, clamps, initial states, materials.

This module generates inputs only.  It holds none of the solver's arithmetic
(no energies, gradients, stiffness fits, matrices or solves), so the CPU oracle
and the CUDA path can both draw their inputs from it without sharing any part
of the method.

Meshes are Kuhn subdivisions of a cube lattice: every cube is split into the six
tetrahedra that share its main diagonal, one per ordering of the three axes.
The paper's own meshes (Table 1) are not available; these lattices stand in for
them with the same element type and comparable tets-per-vertex ratio (~5.6).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

# material kinds, same integer codes as the C header's sim_material_kind
NEOHOOKEAN, STVK, SPLINE_VL, COROTATED, POLY4 = 0, 1, 2, 3, 4
MATERIAL_NAMES = {NEOHOOKEAN: "neohookean", STVK: "stvk", SPLINE_VL: "spline",
                  COROTATED: "corotated", POLY4: "poly4"}

# knots of the synthetic spline materials (principal stretch for a, products for b, c)
SPLINE_KNOTS = (0.3, 0.5, 0.7, 0.85, 1.0, 1.2, 1.6, 2.5)


@dataclass
class Material:
    kind: int
    E: float
    nu: float
    density: float = 1000.0
    # spline control points, shape (3, 8, 3): function (a, b, c) x knot x (x, value, slope)
    spline: np.ndarray | None = None
    # anisotropic fibre term kappa/2 (|F d| - 1)^2 (Sec. 4.4); kappa = 0: none
    kappa: float = 0.0
    fiber: tuple = (0.0, 0.0, 0.0)

    @property
    def mu(self) -> float:
        return self.E / (2.0 * (1.0 + self.nu))

    @property
    def lam(self) -> float:
        return self.E * self.nu / ((1.0 + self.nu) * (1.0 - 2.0 * self.nu))


@dataclass
class Collider:
    """An analytic collider: a plane (point on it, normal pointing to the free
    side), a sphere the body stays outside of (centre, radius) or a torus
    (centre, axis as `normal`, ring radius `major`, tube radius `radius`)."""
    kind: str                     # "plane", "sphere" or "torus"
    point: tuple                  # a point of the plane, or the sphere's / torus's centre
    normal: tuple = (0.0, 0.0, 1.0)
    radius: float = 0.0
    major: float = 0.0

    def as_tuple(self):
        if self.kind == "plane":
            return ("plane", tuple(self.point), tuple(self.normal))
        if self.kind == "torus":
            return ("torus", tuple(self.point), tuple(self.normal), float(self.major), float(self.radius))
        return ("sphere", tuple(self.point), float(self.radius))


@dataclass
class Workload:
    name: str
    rest_pos: np.ndarray          # (n, 3) float64, rest positions X
    tets: np.ndarray              # (T, 4) int32, positively oriented
    clamped: np.ndarray           # (n,) uint8, 1 = position prescribed
    q_cur: np.ndarray             # (n, 3) float64, state q_l
    q_prev: np.ndarray            # (n, 3) float64, state q_{l-1}
    material: Material
    h: float = 1.0 / 30.0
    gravity: tuple = (0.0, 0.0, -9.81)
    iters: int = 10
    history: int = 5
    dims: tuple = ()
    meta: dict = field(default_factory=dict)
    colliders: tuple = ()         # Collider instances
    contact_scale: float = 100.0  # collision weight w_v = contact_scale * m_v / h^2
    # several materials in one mesh: `material` is material 0, these follow it,
    # and tet_material[t] is tet t's index into (material,) + extra_materials
    extra_materials: tuple = ()
    tet_material: np.ndarray | None = None

    @property
    def n_verts(self) -> int:
        return self.rest_pos.shape[0]

    @property
    def n_tets(self) -> int:
        return self.tets.shape[0]


def kuhn_lattice(nx: int, ny: int, nz: int, edge: float = 0.05):
    """Vertices and tets of an nx*ny*nz cube lattice, 6 tets per cube.

    Vertex (i, j, k) has index i + (nx+1)*(j + (ny+1)*k).  Each tet walks from
    the cube's low corner to its high corner along one ordering of the axes;
    odd orderings swap their last two vertices so every tet is positively
    oriented (orientation follows from the permutation's parity alone).
    """
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1),
                             indexing="ij")
    # order vertices by the index formula (k slowest)
    pos = np.zeros(((nx + 1) * (ny + 1) * (nz + 1), 3))
    vid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)
    ids = vid(gi, gj, gk)
    pos[ids.ravel(), 0] = gi.ravel() * edge
    pos[ids.ravel(), 1] = gj.ravel() * edge
    pos[ids.ravel(), 2] = gk.ravel() * edge

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    # cubes ordered with i fastest
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        parity = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b]) % 2
        path = [np.array([0, 0, 0])]
        for ax in perm:
            step = path[-1].copy()
            step[ax] += 1
            path.append(step)
        v = [vid(ci + p[0], cj + p[1], ck + p[2]) for p in path]
        if parity:
            v[2], v[3] = v[3], v[2]
        tets.append(np.stack(v, axis=1))
    # interleave so the 6 tets of one cube are adjacent in memory
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return pos, tets


def _integrate_curvature(x, sig, one, v_one, d_one):
    """Values and slopes at the knots x of the function whose second
    derivative is linear between the knot values sig, with value v_one and
    slope d_one at knot `one` (a C2 cubic spline; cubic Hermite interpolation
    of the returned data reproduces it exactly)."""
    v = np.zeros_like(x)
    d = np.zeros_like(x)
    v[one], d[one] = v_one, d_one
    for i in range(one, x.size - 1):
        h = x[i + 1] - x[i]
        d[i + 1] = d[i] + h * (sig[i] + sig[i + 1]) / 2.0
        v[i + 1] = v[i] + h * d[i] + h * h * (2.0 * sig[i] + sig[i + 1]) / 6.0
    for i in range(one, 0, -1):
        h = x[i] - x[i - 1]
        d[i - 1] = d[i] - h * (sig[i - 1] + sig[i]) / 2.0
        v[i - 1] = v[i] - h * d[i] + h * h * (sig[i - 1] + 2.0 * sig[i]) / 6.0
    return v, d


def spline_control_points(mu: float, lam: float, rng: np.random.Generator,
                          spread: float = 0.3) -> np.ndarray:
    """Control points of a synthetic spline Valanis-Landel material.

    The base is the Neo-Hookean choice a(x) = mu/2 (x^2 - 1), b = 0,
    c(J) = -mu ln J + lam/2 ln^2 J.  At every knot the base curve's second
    derivative (a'' = mu, c'' = (mu + lam - lam ln J) / J^2) is scaled by
    (1 + u), u ~ U[-spread, spread]; values and slopes are the exact
    integrals of that piecewise-linear curvature, anchored at 1 with the base
    values a(1) = c(1) = 0, a'(1) = mu and c'(1) = -a'(1) - 2 b'(1) (a
    stress-free rest state).  So each curve stays within a few tens of percent
    of the Neo-Hookean one and is convex with positive curvature at the end
    knots: the energy is bounded below, as a time step needs.  b stays 0.
    Returns (3, 8, 3): function (a, b, c) x knot x (knot, value, slope).
    """
    k = np.asarray(SPLINE_KNOTS, dtype=np.float64)
    one = int(np.argmin(np.abs(k - 1.0)))
    lk = np.log(k)
    sig_a = mu * (1.0 + rng.uniform(-spread, spread, k.size))
    sig_c = (mu + lam - lam * lk) / (k * k) * (1.0 + rng.uniform(-spread, spread, k.size))
    a_v, a_s = _integrate_curvature(k, sig_a, one, 0.0, mu)
    c_v, c_s = _integrate_curvature(k, sig_c, one, 0.0, -mu)
    out = np.zeros((3, k.size, 3))
    for f, (v, s) in enumerate(((a_v, a_s), (np.zeros_like(k), np.zeros_like(k)), (c_v, c_s))):
        out[f, :, 0] = k
        out[f, :, 1] = v
        out[f, :, 2] = s
    return out


def _with_velocity(rest, clamped, v0, h):
    """States (q_l, q_{l-1}) with q_l = rest and finite-difference velocity v0."""
    q_cur = rest.copy()
    q_prev = rest - h * v0
    q_prev[clamped.astype(bool)] = rest[clamped.astype(bool)]
    return q_cur, q_prev


def lattice_workload(dims, material: Material, *, clamp_axis: int = 2, seed: int = 0,
                     v_range: float = 0.0, v_mode: str = "iid", edge: float = 0.05, iters: int = 10,
                     history: int = 5, gravity=(0.0, 0.0, -9.81), h: float = 1.0 / 30.0,
                     twist_deg: float = 0.0, name: str = "lattice") -> Workload:
    """A Kuhn lattice with its clamp_axis = 0 face clamped (clamp_axis < 0:
    nothing clamped).

    v_range > 0 gives the free vertices an initial velocity with components
    drawn from U[-v_range, v_range]: v_mode "iid" draws every vertex's own
    (a white-noise field that tangles the mesh: a stress input for the
    inverted-element paths), "body" draws one velocity shared by every free
    vertex (the whole body set moving against its clamped face).
    twist_deg rotates the initial state about the long (x) axis by
    twist_deg * x / L.
    """
    nx, ny, nz = dims
    rest, tets = kuhn_lattice(nx, ny, nz, edge)
    if clamp_axis < 0:  # nothing clamped
        clamped = np.zeros(rest.shape[0], dtype=np.uint8)
    else:
        clamped = (np.abs(rest[:, clamp_axis]) < 1e-12 * edge).astype(np.uint8)
    rng = np.random.default_rng(seed)
    v0 = np.zeros_like(rest)
    if v_range > 0.0:
        if v_mode == "iid":
            v0 = rng.uniform(-v_range, v_range, rest.shape)
        elif v_mode == "body":
            v0[:] = rng.uniform(-v_range, v_range, 3)
        else:
            raise ValueError(f"unknown v_mode {v_mode!r}")
        v0[clamped.astype(bool)] = 0.0
    q_cur, q_prev = _with_velocity(rest, clamped, v0, h)
    if twist_deg != 0.0:
        L = nx * edge
        yc, zc = 0.5 * ny * edge, 0.5 * nz * edge
        th = math.radians(twist_deg) * rest[:, 0] / L
        c, s = np.cos(th), np.sin(th)
        dy, dz = rest[:, 1] - yc, rest[:, 2] - zc
        q_cur = rest.copy()
        q_cur[:, 1] = yc + c * dy - s * dz
        q_cur[:, 2] = zc + s * dy + c * dz
        q_prev = q_cur.copy()
    return Workload(name=name, rest_pos=rest, tets=tets, clamped=clamped, q_cur=q_cur,
                    q_prev=q_prev, material=material, h=h, gravity=tuple(gravity),
                    iters=iters, history=history, dims=tuple(dims),
                    meta={"seed": seed, "v_range": v_range, "v_mode": v_mode, "twist_deg": twist_deg})


# ---- the five measured workloads -------------------------------------------------

def bar_4x4x16_fp64() -> Workload:
    """4x4x16 cube bar (1536 tets, 425 vertices), Neo-Hookean E=1e5 nu=0.45, z=0 end clamped."""
    return lattice_workload((4, 4, 16), Material(NEOHOOKEAN, 1e5, 0.45), clamp_axis=2,
                            seed=1604, name="bar4x4x16_nh")


def cube40(kind: int = NEOHOOKEAN, n: int = 40, v_mode: str = "body") -> Workload:
    """n^3 cube lattice (n=40: 384,000 tets, 68,921 vertices), E=5e5 nu=0.4,
    z=0 face clamped, the free vertices set moving with one seeded velocity
    drawn from U[-0.5, 0.5]^3 m/s (v_mode "iid": every vertex's own)."""
    w = lattice_workload((n, n, n), Material(kind, 5e5, 0.4), clamp_axis=2, seed=1605,
                         v_range=0.5, v_mode=v_mode, name=f"cube{n}_{MATERIAL_NAMES[kind]}")
    w.meta["v_mode"] = v_mode
    return w


def spline_bar_80x40x40(scale: int = 1) -> Workload:
    """80x40x40 bar (768,000 tets), synthetic spline VL material, x=0 end clamped,
    initial state twisted 90 degrees along the bar.  scale > 1 divides each
    dimension (small cases for tests)."""
    dims = (80 // scale, 40 // scale, 40 // scale)
    mat = Material(SPLINE_VL, 5e5, 0.4)
    rng = np.random.default_rng(1606)
    mat.spline = spline_control_points(mat.mu, mat.lam, rng)
    return lattice_workload(dims, mat, clamp_axis=0, seed=1606, twist_deg=90.0,
                            name=f"splinebar{dims[0]}x{dims[1]}x{dims[2]}")


def fiber_cube(n: int = 8, kappa_scale: float = 5.0, fiber=(1.0, 1.0, 0.0), v: float = 0.5) -> Workload:
    """Sec. 4.4's anisotropic example: an n^3 cube of corotated material
    (mu : lambda = 1 : 10, as in the paper's mu = 10, lambda = 100) reinforced
    along `fiber` with kappa = kappa_scale * mu (the paper's 50 = 5 mu),
    z = 0 face clamped, the free vertices set moving with one seeded velocity
    drawn from U[-v, v]^3 m/s."""
    nu = 10.0 / 22.0                  # lambda / mu = 2 nu / (1 - 2 nu) = 10
    E = 2.0 * (1.0 + nu) * 2e4        # mu = 2e4 Pa
    mat = Material(COROTATED, E, nu)
    d = np.asarray(fiber, dtype=np.float64)
    mat.fiber = tuple(d / np.linalg.norm(d))
    mat.kappa = kappa_scale * mat.mu
    return lattice_workload((n, n, n), mat, clamp_axis=2, seed=1610, v_range=v, v_mode="body",
                            name=f"fibercube{n}")


def collision_drop(n: int = 8, drop: float = 0.02, speed: float = 2.0, sphere: bool = True,
                   kind: int = NEOHOOKEAN, E: float = 2e5, name: str = "", torus: bool = False) -> Workload:
    """An unclamped n^3 Neo-Hookean cube falling onto the ground plane z = 0
    (Sec. 4.3's collision terms), its lowest face `drop` above it, every
    vertex moving down at `speed` m/s; with `sphere`, a sphere of radius
    n*edge/4, sunk into the ground so that its top is just below the cube,
    sits under one corner of the cube's footprint: that corner lands on it
    first.  With `torus`, a ring (axis z, centred under the cube, ring
    radius n*edge/4, tube radius n*edge/8) lies sunk into the ground with
    its top just below the cube, in place of the sphere: the vertices above
    the ring land on its tube first."""
    edge = 0.05
    w = lattice_workload((n, n, n), Material(kind, E, 0.4), clamp_axis=-1, seed=1609, name=name or f"drop{n}")
    shift = np.array([-0.5 * n * edge, -0.5 * n * edge, drop])
    v = np.array([0.0, 0.0, -speed])
    w.q_cur = w.rest_pos + shift
    w.q_prev = w.q_cur - w.h * v
    cols = [Collider("plane", (0.0, 0.0, 0.0), (0.0, 0.0, 1.0))]
    if torus:
        r = n * edge / 8.0
        top = 0.5 * drop
        cols.append(Collider("torus", (0.0, 0.0, top - r), (0.0, 0.0, 1.0), radius=r, major=n * edge / 4.0))
    elif sphere:
        r = 0.25 * n * edge
        top = 0.5 * drop  # the sphere's top, between the ground and the cube
        cols.append(Collider("sphere", (-0.25 * n * edge, -0.25 * n * edge, top - r), radius=r))
    w.colliders = tuple(cols)
    w.meta.update({"drop": drop, "speed": speed})
    return w


def batch_512(count: int = 512, lo: int = 4, hi: int = 24, seed: int = 1607) -> list:
    """Independent simulations: per-axis dims uniform in [lo, hi], material uniform
    over {Neo-Hookean, StVK, spline}, E log-uniform in [1e4, 1e6], nu ~ U[0.3, 0.48],
    x=0 face clamped, gravity, zero initial velocity."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        dims = tuple(int(d) for d in rng.integers(lo, hi + 1, size=3))
        kind = (NEOHOOKEAN, STVK, SPLINE_VL)[int(rng.integers(0, 3))]
        E = float(10.0 ** rng.uniform(4.0, 6.0))
        nu = float(rng.uniform(0.3, 0.48))
        mat = Material(kind, E, nu)
        if kind == SPLINE_VL:
            mat.spline = spline_control_points(mat.mu, mat.lam, rng)
        out.append(lattice_workload(dims, mat, clamp_axis=0, seed=seed + 1 + s,
                                    name=f"batch{s}"))
    return out


def large_48x48x192() -> Workload:
    """48x48x192 bar (2,654,208 tets, 463,393 vertices), Neo-Hookean E=5e5 nu=0.4,
    z=0 end clamped, a seeded impulse: one velocity drawn from U[-0.5, 0.5]^3 m/s
    for every free vertex, 20 iterations, m=8."""
    return lattice_workload((48, 48, 192), Material(NEOHOOKEAN, 5e5, 0.4), clamp_axis=2,
                            seed=1608, v_range=0.5, v_mode="body", iters=20, history=8,
                            name="bar48x48x192_nh")


def two_material_bar(dims, mat_a: Material, mat_b: Material, *, seed: int = 0, v_range: float = 0.0,
                     v_mode: str = "body", name: str = "two_material") -> Workload:
    """A Kuhn lattice (z = 0 face clamped) whose tets with centroid x below
    half the bar's length take mat_a and the others mat_b."""
    w = lattice_workload(dims, mat_a, seed=seed, v_range=v_range, v_mode=v_mode, name=name)
    cx = w.rest_pos[w.tets].mean(axis=1)[:, 0]
    w.extra_materials = (mat_b,)
    w.tet_material = (cx >= 0.5 * dims[0] * 0.05).astype(np.int32)
    return w
