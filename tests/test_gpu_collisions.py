"""Collision terms (Sec. 4.3) on the GPU against the oracle: a cube falling
onto a ground plane and a sphere, or a ground plane and a torus.  The active set is decided per vertex at
the start of every iteration in both; FP64 is held to round-off, FP32 to the
method's position tolerance."""
import numpy as np
import pytest

from oracle import hqn_oracle as O
from paper_1604_07378_gb300 import workloads as W

from _util import problem_for, rel, sim_for

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07378_gb300 import hqn
    hqn.library()


def _in_contact(n=4):
    """The drop workload advanced (by the oracle) until the cube presses on
    the plane and the sphere."""
    w = W.collision_drop(n, drop=0.004, speed=2.0)
    P = problem_for(w)
    qc, qp = w.q_cur.copy(), w.q_prev.copy()
    for _ in range(2):
        x, _ = O.solve_step(P, qc, qp, iters=10, m=5)
        qp, qc = qc, x
    return w, P, qc, qp


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_energy_gradient_with_contacts(prec):
    w, P, qc, qp = _in_contact()
    y = O.predictor(P, qc, qp)
    x = qc + 0.5 * (y - qc)
    C = O.contact_terms(P, x, qc)
    assert C.idx.size > 10
    g_ref = O.objective(P, x, y, C)
    grad_ref = O.gradient(P, x, y, C)
    with sim_for(w, prec, use_graph=0) as sim:
        sim.set_state(qc, qp)
        g, grad = sim.energy_grad(x, y)
    assert rel(grad, grad_ref) <= (1e-11 if prec == FP64 else 1e-5), rel(grad, grad_ref)
    assert abs(g - g_ref) <= (1e-11 if prec == FP64 else 2e-6) * abs(g_ref)


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("use_graph", [1, 0], ids=["graph", "eager"])
def test_step_with_contacts_matches_oracle(prec, use_graph):
    w, P, qc, qp = _in_contact()
    x_ref, st = O.solve_step(P, qc, qp, iters=w.iters, m=w.history)
    with sim_for(w, prec, use_graph=use_graph) as sim:
        sim.set_state(qc, qp)
        rc, stats = sim.step(1, stats=True)
        x, _ = sim.get_state()
    assert rc >= 0
    assert rel(x, x_ref) <= (1e-9 if prec == FP64 else 1e-4), rel(x, x_ref)
    if prec == FP64:
        assert stats["trials"] == st.trials
        np.testing.assert_allclose(stats["g"], st.g, rtol=1e-9)


def test_drop_trajectory_fp64():
    """Twelve steps of the fall from above the colliders through the impact,
    along the oracle's trajectory: every GPU step, started from the oracle's
    state, matches the oracle's step (positions, trial counts and objective
    values).  Steps are compared one at a time because the contact dynamics
    amplify round-off over a long free-running trajectory: a borderline
    Armijo test can then choose another step length."""
    w = W.collision_drop(4, drop=0.01, speed=2.0)
    P = problem_for(w)
    qc, qp = w.q_cur.copy(), w.q_prev.copy()
    with sim_for(w, FP64) as sim:
        for k in range(12):
            x_ref, st = O.solve_step(P, qc, qp, iters=w.iters, m=w.history)
            sim.set_state(qc, qp)
            rc, stats = sim.step(1, stats=True)
            x, _ = sim.get_state()
            assert rc >= 0
            assert rel(x, x_ref) <= 1e-9, (k, rel(x, x_ref))
            assert stats["trials"] == st.trials, k
            np.testing.assert_allclose(stats["g"], st.g, rtol=1e-9)
            qp, qc = qc, x_ref
    assert qc[:, 2].min() < 0.0  # the cube did reach the ground


def test_batch_with_contacts_bitwise_equal_to_single_handles():
    """The colliders are shared by a batch's simulations (they are part of the
    parameters): every single handle gets the batch's colliders."""
    from paper_1604_07378_gb300 import hqn
    ws = [W.collision_drop(n, drop=0.004, speed=s) for n, s in ((3, 2.0), (4, 1.0), (5, 1.5))]
    cols = ws[0].colliders
    with hqn.Batch(ws, precision=FP32) as b:
        for i, w in enumerate(ws):
            b.set_state(i, w.q_cur, w.q_prev)
        b.step(4)
        got = [b.get_state(i)[0] for i in range(len(ws))]
    for i, w in enumerate(ws):
        with hqn.Sim.from_workload(w, precision=FP32, colliders=cols) as sim:
            sim.set_state(w.q_cur, w.q_prev)
            sim.step(4)
            np.testing.assert_array_equal(got[i], sim.get_state()[0])


def _on_torus():
    """The drop onto the ring (in place of the sphere), advanced by the oracle
    until vertices press on the torus tube."""
    w = W.collision_drop(4, drop=0.004, speed=2.0, torus=True)
    P = problem_for(w)
    qc, qp = w.q_cur.copy(), w.q_prev.copy()
    for _ in range(2):
        x, _ = O.solve_step(P, qc, qp, iters=10, m=5)
        qp, qc = qc, x
    return w, P, qc, qp


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_torus_contacts_energy_gradient_and_step(prec):
    """Contacts with a torus (the ground plane and a ring, Sec. 4.3's
    examples): g and its gradient at a point between the state and the
    predictor, then one whole step, against the oracle."""
    w, P, qc, qp = _on_torus()
    y = O.predictor(P, qc, qp)
    x = qc + 0.5 * (y - qc)
    C = O.contact_terms(P, x, qc)
    assert np.sum(np.abs(C.n[:, 2]) < 0.999) > 0  # some normals are the tube's
    g_ref, grad_ref = O.objective(P, x, y, C), O.gradient(P, x, y, C)
    x_ref, st = O.solve_step(P, qc, qp, iters=w.iters, m=w.history)
    with sim_for(w, prec) as sim:
        sim.set_state(qc, qp)
        g, grad = sim.energy_grad(x, y)
        rc, stats = sim.step(1, stats=True)
        xs, _ = sim.get_state()
    assert rel(grad, grad_ref) <= (1e-11 if prec == FP64 else 1e-5), rel(grad, grad_ref)
    assert abs(g - g_ref) <= (1e-11 if prec == FP64 else 2e-6) * abs(g_ref)
    assert rc >= 0
    assert rel(xs, x_ref) <= (1e-9 if prec == FP64 else 1e-4), rel(xs, x_ref)
    if prec == FP64:
        assert stats["trials"] == st.trials


def test_torus_parameters_are_checked():
    from paper_1604_07378_gb300 import hqn
    w = W.collision_drop(2, torus=True)
    bad = W.Collider("torus", (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), radius=0.2, major=0.1)  # tube wider than the ring
    with pytest.raises(hqn.HQNError) as e:
        sim_for(w, FP32, colliders=(bad,))
    assert e.value.code == hqn.HQN_ERR_ARG


# ---------------------------------------------------------------- anisotropic fibre term (Sec. 4.4)

def _fiber_workloads():
    w_cor = W.fiber_cube(4)                                  # corotated base (signed-SVD path)
    w_nh = W.fiber_cube(4, fiber=(0.0, 1.0, 1.0))
    w_nh.material.kind = W.NEOHOOKEAN                        # invariant-form base
    return [w_cor, w_nh]


@pytest.mark.parametrize("idx", [0, 1], ids=["corotated", "neohookean"])
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_fiber_energy_gradient_and_step(idx, prec):
    w = _fiber_workloads()[idx]
    P = problem_for(w)
    y = O.predictor(P, w.q_cur, w.q_prev)
    rng = np.random.default_rng(21)
    x = y + 3e-3 * rng.normal(size=y.shape) * (~w.clamped.astype(bool))[:, None]
    x_ref, st = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history)
    with sim_for(w, prec) as sim:
        g, grad = sim.energy_grad(x, y)
        sim.set_state(w.q_cur, w.q_prev)
        rc, stats = sim.step(1, stats=True)
        xs, _ = sim.get_state()
    assert rel(grad, O.gradient(P, x, y)) <= (1e-10 if prec == FP64 else 1e-5)
    assert abs(g - O.objective(P, x, y)) <= (1e-10 if prec == FP64 else 2e-6) * abs(O.objective(P, x, y))
    assert rc >= 0
    assert rel(xs, x_ref) <= (1e-9 if prec == FP64 else 1e-4), rel(xs, x_ref)
    if prec == FP64:
        assert stats["trials"] == st.trials
