"""Jacobi-PCG in lieu of the factorised A0^{-1} (the paper's comparison with
iterative solvers): the GPU's matrix-free PCG against the oracle's, alone and
inside whole steps."""
import numpy as np
import pytest

from oracle import hqn_oracle as O
from paper_1604_07378_gb300 import workloads as W

from _util import perturbed, problem_for, rel, sim_for, small_workloads

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1
WORKLOADS = small_workloads()
IDS = [w.name for w in WORKLOADS]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_07378_gb300 import hqn
    hqn.library()


@pytest.mark.parametrize("iters", [1, 5, 15])
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_pcg_solve_matches_oracle(iters, prec):
    w = WORKLOADS[1]
    P = problem_for(w)
    rng = np.random.default_rng(30 + iters)
    q = rng.normal(size=(w.n_verts, 3))
    with sim_for(w, prec, use_graph=0, a0_solver=1, pcg_iters=iters) as sim:
        r = sim.solve_A0(q)
    r_ref = O.solve_A_pcg(P, q, iters)
    assert rel(r, r_ref) <= (1e-11 if prec == FP64 else 1e-5), rel(r, r_ref)
    assert np.all(r[w.clamped.astype(bool)] == 0.0)


@pytest.mark.parametrize("w", WORKLOADS, ids=IDS)
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_step_with_pcg_matches_oracle(w, prec):
    P = problem_for(w)
    x_ref, st = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history, pcg_iters=15)
    with sim_for(w, prec, use_graph=1, a0_solver=1, pcg_iters=15) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        rc, stats = sim.step(1, stats=True)
        x, _ = sim.get_state()
    assert rc >= 0
    assert rel(x, x_ref) <= (1e-9 if prec == FP64 else 1e-4), rel(x, x_ref)
    if prec == FP64:
        assert stats["trials"] == st.trials


# ---------------------------------------------------------------- Chebyshev direction (Alg. 3)

@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_chebyshev_step_matches_oracle(prec):
    """30 iterations on the twisting spline bar with the Chebyshev direction
    (S = 10, rho = 0.99): the acceleration is active for the last 20."""
    w = W.spline_bar_80x40x40(scale=10)
    P = problem_for(w)
    x_ref, st = O.solve_step(P, w.q_cur, w.q_prev, iters=30, chebyshev=(10, 0.99))
    with sim_for(w, prec, use_graph=1, iters=30, direction=1, cheb_S=10, cheb_rho=0.99) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        rc, stats = sim.step(1, stats=True)
        x, _ = sim.get_state()
    assert rc >= 0
    assert rel(x, x_ref) <= (1e-9 if prec == FP64 else 1e-4), rel(x, x_ref)
    if prec == FP64:
        assert stats["trials"][:30] == st.trials
        np.testing.assert_allclose(stats["g"][:30], st.g, rtol=1e-10)
