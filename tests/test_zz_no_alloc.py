"""The allocation-free entry point hqn_energy_grad_static against sim_energy_grad.

hqn_energy_grad_static serves callers that cannot allocate device memory
(code inside a memory pool or budget that someone else owns, plug-ins that
must not call the CUDA allocator, drivers that forbid cudaMalloc while they
run): its scratch is a fixed array that the library keeps in each GPU's
memory.  These tests call it through the C ABI on device buffers and compare
g and grad g with what a float64 handle's sim_energy_grad returns for the
same x and y, within the float64 tolerance of the other parity tests.  Two
calls in a row on different states check that the shared scratch carries
nothing wrong from one call to the next.

The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1604_07378_gb300 import workloads as W

from _util import perturbed, rel


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
    y = w.q_cur.copy()
    with hqn.Sim.from_workload(w, precision=hqn.FP64_PLAIN, use_graph=0) as sim:
        for call, (scale, seed) in enumerate(((4e-3, 1), (1.5e-2, 2))):
            x = perturbed(w, scale, seed)
            g_ref, grad_ref = sim.energy_grad(x, y)
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
            assert np.all(grad_h[w.clamped.astype(bool)] == 0.0)
