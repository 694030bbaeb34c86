"""The allocation-free entry point hqn_energy_grad_static against the FP64
oracle and against sim_energy_grad.

hqn_energy_grad_static serves callers that cannot allocate device memory
(code inside a memory pool or budget that someone else owns, plug-ins that
must not call the CUDA allocator, drivers that forbid cudaMalloc while they
run): its scratch is a fixed array that the library keeps in each GPU's
memory.  These tests call it through the C ABI on device buffers and compare
g and grad g with the oracle's objective and gradient (Eq. PD) and with what
a float64 handle's sim_energy_grad returns for the same x and y, within the
float64 tolerance of the other parity tests.  The states move the clamped
vertices too (x != y there), which the inertia term must skip.  Two calls in
a row on different states check that the shared scratch carries nothing
wrong from one call to the next.

The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import hqn_oracle as O
from paper_1604_07378_gb300 import workloads as W

from _util import rel


def _csr(tets, n):
    """Incident-corner lists (4 * tet + corner) of every vertex, ascending tet."""
    T = tets.shape[0]
    slot = (4 * np.arange(T)[:, None] + np.arange(4)[None, :]).ravel()
    vert = tets.ravel()
    order = np.argsort(vert, kind="stable")
    ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(ptr, vert + 1, 1)
    return np.cumsum(ptr).astype(np.int32), slot[order].astype(np.int32)


def _material(m):
    from paper_1604_07378_gb300 import hqn
    spline = None if m.spline is None else np.ascontiguousarray(m.spline, dtype=np.float64)
    mat = hqn.Material(m.kind, m.E, m.nu, m.density,
                       None if spline is None else spline.ctypes.data_as(C.POINTER(C.c_double)))
    return mat, spline


def test_rejects_meshes_beyond_the_scratch_capacity():
    """Checked before any device work, so no GPU is needed."""
    from paper_1604_07378_gb300 import hqn
    lib = hqn.library()
    w = W.lattice_workload((2, 2, 2), W.Material(W.NEOHOOKEAN, 1e5, 0.45))
    mat, _ = _material(w.material)
    rc = lib.hqn_energy_grad_static(w.n_verts, hqn.STATIC_MAX_TETS + 1, None, None, None, None, None,
                                    C.byref(mat), w.h, None, None, None, None, None)
    assert rc == hqn.HQN_ERR_ARG
    assert b"exceed the static scratch capacity" in lib.hqn_last_error()


@pytest.mark.parametrize("E,nu,density", [(1e5, 0.5, 1000.0), (0.0, 0.3, 1000.0), (-1e5, 0.3, 1000.0),
                                          (1e5, -1.0, 1000.0), (1e5, 0.3, 0.0)])
def test_rejects_bad_materials(E, nu, density):
    """The material is checked as sim_create checks it, before any device
    work (the device pointers below are never dereferenced): nu = 0.5 would
    make lambda infinite, E <= 0 or density <= 0 meaningless."""
    from paper_1604_07378_gb300 import hqn
    lib = hqn.library()
    w = W.lattice_workload((2, 2, 2), W.Material(W.NEOHOOKEAN, 1e5, 0.45))
    mat = hqn.Material(W.NEOHOOKEAN, E, nu, density, None)
    fake = 256  # a non-null stand-in for each device array
    rc = lib.hqn_energy_grad_static(w.n_verts, w.n_tets, fake, fake, fake, fake, fake, C.byref(mat), w.h,
                                    fake, fake, fake, fake, None)
    assert rc == hqn.HQN_ERR_ARG
    assert lib.hqn_last_error().startswith(b"hqn_energy_grad_static")


def _moved_state(w, scale, seed):
    """A seeded state that moves every vertex, the clamped ones included."""
    rng = np.random.default_rng(seed)
    return w.q_cur + scale * rng.normal(size=w.q_cur.shape)


@pytest.mark.gpu
@pytest.mark.parametrize("kind", [W.NEOHOOKEAN, W.STVK, W.SPLINE_VL])
def test_static_energy_grad_matches_sim_energy_grad(kind):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07378_gb300 import hqn
    lib = hqn.library()
    mat = W.Material(kind, 5e5, 0.4)
    if kind == W.SPLINE_VL:
        mat.spline = W.spline_control_points(mat.mu, mat.lam, np.random.default_rng(3))
    # several blocks of both kernels and a ragged tail (1,890 tets, 448 vertices)
    w = W.lattice_workload((5, 7, 9), mat, clamp_axis=2, seed=21, v_range=0.5)
    assert w.n_tets <= hqn.STATIC_MAX_TETS
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    vt_ptr, vt_slot = _csr(w.tets, w.n_verts)
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    X = d(w.rest_pos, torch.float64)
    tets = d(w.tets, torch.int32)
    clamped = d(w.clamped, torch.uint8)
    ptr, slot = d(vt_ptr, torch.int32), d(vt_slot, torch.int32)
    cmat, _keep = _material(w.material)
    P = O.problem_from_workload(w)
    y = O.predictor(P, w.q_cur, w.q_prev)
    with hqn.Sim.from_workload(w, precision=hqn.FP64_PLAIN, use_graph=0) as sim:
        for call, (scale, seed) in enumerate(((4e-3, 1), (1.5e-2, 2))):
            x = _moved_state(w, scale, seed)
            g_ref, grad_ref = O.objective(P, x, y), O.gradient(P, x, y)
            g_sim, grad_sim = sim.energy_grad(x, y)
            xd, yd = d(x, torch.float64), d(y, torch.float64)
            g = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            grad = torch.full((w.n_verts, 3), float("nan"), dtype=torch.float64, device=dev)
            rc = lib.hqn_energy_grad_static(
                w.n_verts, w.n_tets, X.data_ptr(), tets.data_ptr(), clamped.data_ptr(), ptr.data_ptr(),
                slot.data_ptr(), C.byref(cmat), w.h, xd.data_ptr(), yd.data_ptr(), g.data_ptr(),
                grad.data_ptr(), stream.cuda_stream)
            assert rc == hqn.HQN_OK, lib.hqn_last_error()
            torch.cuda.synchronize()
            g_h, grad_h = float(g.item()), grad.cpu().numpy()
            assert abs(g_h - g_ref) <= 1e-11 * abs(g_ref), (call, g_h, g_ref)
            assert rel(grad_h, grad_ref) <= 1e-11, (call, rel(grad_h, grad_ref))
            assert abs(g_h - g_sim) <= 1e-11 * abs(g_ref), (call, g_h, g_sim)
            assert rel(grad_h, grad_sim) <= 1e-11, (call, rel(grad_h, grad_sim))
            assert np.all(grad_h[w.clamped.astype(bool)] == 0.0)


@pytest.mark.gpu
def test_static_energy_grad_out_of_range_indices_give_nan():
    """A tet index one past the vertex arrays, or a corner slot one past
    the corner array, is not dereferenced: the call returns NaN for g (and
    the affected gradient rows) and the next well-formed call is exact."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07378_gb300 import hqn
    lib = hqn.library()
    w = W.lattice_workload((3, 3, 4), W.Material(W.NEOHOOKEAN, 5e5, 0.4), seed=4, v_range=0.3)
    P = O.problem_from_workload(w)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    vt_ptr, vt_slot = _csr(w.tets, w.n_verts)
    cmat, _keep = _material(w.material)
    x = _moved_state(w, 3e-3, 5)
    y = O.predictor(P, w.q_cur, w.q_prev)
    X, xd, yd, cl = d(w.rest_pos, torch.float64), d(x, torch.float64), d(y, torch.float64), d(w.clamped, torch.uint8)
    bad_tets = w.tets.copy()
    bad_tets[7, 2] = w.n_verts
    bad_slot = vt_slot.copy()
    v_free = int(np.flatnonzero(w.clamped == 0)[0])  # a clamped vertex's gradient row is zero anyway
    bad_slot[vt_ptr[v_free]] = 4 * w.n_tets
    cases = ((bad_tets, vt_slot, False), (w.tets, bad_slot, False), (w.tets, vt_slot, True))
    for tets, slot, good in cases:
        g = torch.zeros(1, dtype=torch.float64, device=dev)
        grad = torch.zeros((w.n_verts, 3), dtype=torch.float64, device=dev)
        td, pd, sd = d(tets, torch.int32), d(vt_ptr, torch.int32), d(slot, torch.int32)
        rc = lib.hqn_energy_grad_static(w.n_verts, w.n_tets, X.data_ptr(), td.data_ptr(), cl.data_ptr(),
                                        pd.data_ptr(), sd.data_ptr(), C.byref(cmat), w.h, xd.data_ptr(),
                                        yd.data_ptr(), g.data_ptr(), grad.data_ptr(), stream.cuda_stream)
        assert rc == hqn.HQN_OK
        torch.cuda.synchronize()
        if good:
            assert abs(float(g.item()) - O.objective(P, x, y)) <= 1e-11 * abs(O.objective(P, x, y))
            assert rel(grad.cpu().numpy(), O.gradient(P, x, y)) <= 1e-11
        else:
            assert np.isnan(float(g.item()))
            assert np.isnan(grad.cpu().numpy()).any()
