"""Batches of independent simulations (sim_batch_create) against the FP64
oracle and against single-simulation handles.

A simulation in a batch owns whole blocks of every kernel, its own reductions
and its own solve items, so its arithmetic is exactly that of a handle made
for it alone: the batch must agree bit for bit with single handles, and each
simulation with the oracle within the usual tolerances.  The batch mixes
mesh sizes, materials and a tangled initial state whose line search
backtracks while the others accept the first trial, so simulations finish
their iterations at different times.
"""
import numpy as np
import pytest

from oracle import hqn_oracle as O
from paper_1604_07378_gb300 import workloads as W

from _util import problem_for, rel

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07378_gb300 import hqn
    hqn.library()


def _batch_workloads():
    rng = np.random.default_rng(31)
    out = []
    mats = [W.Material(W.NEOHOOKEAN, 2e5, 0.4), W.Material(W.STVK, 5e5, 0.35),
            W.Material(W.SPLINE_VL, 3e5, 0.42), W.Material(W.NEOHOOKEAN, 1e6, 0.45),
            W.Material(W.STVK, 8e4, 0.3)]
    for k, mat in enumerate(mats):
        if mat.kind == W.SPLINE_VL:
            mat.spline = W.spline_control_points(mat.mu, mat.lam, rng)
        dims = tuple(int(d) for d in rng.integers(2, 7, size=3))
        out.append(W.lattice_workload(dims, mat, clamp_axis=0, seed=40 + k, v_range=0.3, v_mode="body",
                                      name=f"b{k}"))
    # a tangled state: per-vertex velocities make the line search backtrack
    out.append(W.lattice_workload((4, 3, 5), W.Material(W.NEOHOOKEAN, 5e5, 0.4), clamp_axis=2, seed=47,
                                  v_range=0.5, name="tangled"))
    return out


WL = _batch_workloads()


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("use_graph", [1, 0], ids=["graph", "eager"])
def test_batch_step_matches_oracle_and_single_handles(prec, use_graph):
    from paper_1604_07378_gb300 import hqn
    with hqn.Batch(WL, precision=prec, use_graph=use_graph) as b:
        assert b.info()["n_sims"] == len(WL)
        for i, w in enumerate(WL):
            b.set_state(i, w.q_cur, w.q_prev)
        rc, tot = b.step(1)
        assert rc >= 0
        got = [b.get_state(i)[0] for i in range(len(WL))]
        per = [b.stats(i) for i in range(len(WL))]
    assert tot["trials_total"] == sum(p["trials_total"] for p in per)
    assert max(p["trials_total"] for p in per) > min(p["trials_total"] for p in per)  # uneven searches
    for i, w in enumerate(WL):
        x_ref, st = O.solve_step(problem_for(w), w.q_cur, w.q_prev, iters=w.iters, m=w.history)
        assert rel(got[i], x_ref) <= (1e-9 if prec == FP64 else 1e-4), (i, rel(got[i], x_ref))
        if prec == FP64:
            assert per[i]["trials"] == st.trials, i
        with hqn.Sim.from_workload(w, precision=prec, use_graph=use_graph) as sim:
            sim.set_state(w.q_cur, w.q_prev)
            sim.step(1)
            np.testing.assert_array_equal(got[i], sim.get_state()[0])


def test_batch_several_steps_bitwise_equal_to_single_handles():
    from paper_1604_07378_gb300 import hqn
    with hqn.Batch(WL, precision=FP32) as b:
        for i, w in enumerate(WL):
            b.set_state(i, w.q_cur, w.q_prev)
        b.step(3)
        got = [b.get_state(i) for i in range(len(WL))]
    for i, w in enumerate(WL):
        with hqn.Sim.from_workload(w, precision=FP32) as sim:
            sim.set_state(w.q_cur, w.q_prev)
            sim.step(3)
            qc, qp = sim.get_state()
        np.testing.assert_array_equal(got[i][0], qc)
        np.testing.assert_array_equal(got[i][1], qp)


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_batch_other_sweep_shapes_bitwise_equal_to_single_handles(prec):
    """With other sweep shapes (512-thread blocks, small work items, no L2
    prefetch, each simulation's top two levels in a dense block) each
    simulation's items and tiles are still its own, so the batch agrees bit
    for bit with single handles of the same shapes (and with the oracle)."""
    from paper_1604_07378_gb300 import hqn
    shapes = dict(solve_threads=512, solve_item_kb=16, solve_items=64, solve_prefetch=-1, solve_dense_top=2)
    with hqn.Batch(WL, precision=prec, **shapes) as b:
        info = b.info()
        assert (info["solve_threads"], info["solve_item_kb"], info["solve_prefetch"]) == (512, 16, 0)
        assert info["dense_top_cols"] > 0
        for i, w in enumerate(WL):
            b.set_state(i, w.q_cur, w.q_prev)
        rc, _ = b.step(2)
        assert rc >= 0
        got = [b.get_state(i)[0] for i in range(len(WL))]
    for i, w in enumerate(WL):
        with hqn.Sim.from_workload(w, precision=prec, **shapes) as sim:
            sim.set_state(w.q_cur, w.q_prev)
            sim.step(2)
            np.testing.assert_array_equal(got[i], sim.get_state()[0])
    w = WL[0]
    P = problem_for(w)
    x1, _ = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history)
    x2, _ = O.solve_step(P, x1, w.q_cur, iters=w.iters, m=w.history)
    assert rel(got[0], x2) <= (1e-9 if prec == FP64 else 1e-4)
