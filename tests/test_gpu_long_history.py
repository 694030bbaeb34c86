"""L-BFGS windows longer than 16 pairs (Alg. 2 with m up to 128; the paper's
convergence study of Sec. 5 runs m = 100) against the FP64 oracle.

Windows above 16 pairs keep the two loops' scalars in device memory and form
the slot products in chunks of 16 slots, so these cases cover the chunk
boundaries, the ring's wrap-around once the window is full, and the
per-simulation scalars of a batch."""
import numpy as np
import pytest

from oracle import hqn_oracle as O
from paper_1604_07378_gb300 import workloads as W

from _util import problem_for, rel, sim_for, small_workloads

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1
WORKLOADS = small_workloads()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pairs(P, w, npairs, rng):
    free = ~w.clamped.astype(bool)
    out = []
    for _ in range(npairs):
        s = rng.normal(size=(w.n_verts, 3)) * free[:, None]
        t = np.zeros_like(s)
        t[free] = P.A @ s[free] + 0.01 * rng.normal(size=s[free].shape) * np.abs(P.A @ s[free]).mean()
        out.append((s, t, float(np.sum(s * t))))
    return out


@pytest.mark.parametrize("npairs", [17, 33, 100], ids=["17", "33", "100"])
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_long_direction_parity(npairs, prec):
    """Caller-given pairs, m = 100: the two-loop direction against the
    oracle's Alg. 2 (the pairs span one, two and seven 16-slot chunks)."""
    w = WORKLOADS[1]
    P = problem_for(w)
    rng = np.random.default_rng(100 + npairs)
    free = ~w.clamped.astype(bool)
    grad = rng.normal(size=(w.n_verts, 3)) * free[:, None]
    pairs = _pairs(P, w, npairs, rng)
    d_ref = O.lbfgs_direction(P, grad, pairs)
    with sim_for(w, prec, use_graph=0, history_m=100) as sim:
        d = sim.direction(grad, [p[0] for p in pairs], [p[1] for p in pairs])
    assert rel(d, d_ref) <= (1e-10 if prec == FP64 else 1e-4)


STEP_TOL = {FP64: 1e-8, FP32: 1e-3}


@pytest.mark.parametrize("m,iters", [(100, 30), (20, 40)], ids=["m100", "m20_wraps"])
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("use_graph", [0, 1], ids=["eager", "graph"])
def test_long_window_step_parity(m, iters, prec, use_graph):
    """One step of `iters` iterations with a window of m pairs: m = 100
    holds every pair of the step; m = 20 fills its ring and wraps."""
    w = WORKLOADS[2]
    P = problem_for(w)
    x_ref, st = O.solve_step(P, w.q_cur, w.q_prev, iters=iters, m=m)
    with sim_for(w, prec, use_graph=use_graph, history_m=m, iters=iters) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        rc, stats = sim.step(1, stats=True)
        qc, _ = sim.get_state()
    assert rc >= 0 and stats["iters"] == iters
    assert rel(qc, x_ref) <= (1e-9 if prec == FP64 else 1e-4)
    ex_step = float(np.linalg.norm(qc - x_ref) / np.linalg.norm(x_ref - w.q_cur))
    assert ex_step <= STEP_TOL[prec], ex_step
    if prec == FP64:
        assert stats["trials"] == st.trials
        np.testing.assert_allclose(stats["g"], st.g, rtol=1e-9)


def test_long_window_batch_matches_oracle():
    """Three simulations of different sizes in one handle, m = 24 over 30
    iterations: each simulation's window lives in its own scalars."""
    from paper_1604_07378_gb300 import hqn
    ws = [W.lattice_workload(d, W.Material(W.NEOHOOKEAN, 3e5, 0.4), clamp_axis=0, seed=20 + k, v_range=0.4)
          for k, d in enumerate(((4, 4, 6), (6, 5, 5), (3, 7, 4)))]
    with hqn.Batch(ws, precision=FP64, history_m=24, iters=30) as b:
        for i, w in enumerate(ws):
            b.set_state(i, w.q_cur, w.q_prev)
        rc, _ = b.step(1)
        got = [b.get_state(i)[0] for i in range(len(ws))]
    assert rc >= 0
    for w, x in zip(ws, got):
        x_ref, _ = O.solve_step(problem_for(w), w.q_cur, w.q_prev, iters=30, m=24)
        assert rel(x, x_ref) <= 1e-9, rel(x, x_ref)
