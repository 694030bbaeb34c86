"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances follow the accuracy targets of the method's FP32 form: gradient
relative error <= 1e-5 and per-step position relative error <= 1e-4 after the
step's fixed iterations, both against the FP64 oracle fed the same state.
The FP64 form is held to round-off-level agreement.
"""
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


# ---------------------------------------------------------------- energy and gradient

@pytest.mark.parametrize("w", WORKLOADS, ids=IDS)
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_energy_gradient_parity(w, prec):
    P = problem_for(w)
    y = O.predictor(P, w.q_cur, w.q_prev)
    tol_g = 1e-11 if prec == FP64 else 1e-5
    with sim_for(w, prec, use_graph=0) as sim:
        for seed, scale in ((0, 0.0), (1, 2e-3), (2, 8e-3)):
            x = perturbed(w, scale, seed) if scale else w.q_cur
            g_ref = O.objective(P, x, y)
            grad_ref = O.gradient(P, x, y)
            g, grad = sim.energy_grad(x, y)
            if np.linalg.norm(grad_ref) > 0:
                assert rel(grad, grad_ref) <= tol_g, (seed, rel(grad, grad_ref))
            assert abs(g - g_ref) <= (1e-11 if prec == FP64 else 2e-6) * max(abs(g_ref), 1e-12)
            # clamped rows are exactly zero
            assert np.all(grad[w.clamped.astype(bool)] == 0.0)


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_energy_gradient_clamped_rows_moved(prec):
    """x != y on clamped rows: the clamped vertices are eliminated, so the
    inertia term of Eq. PD skips them (their x still enters the elastic
    energy of their tets) and their gradient rows are zero."""
    w = WORKLOADS[1]
    P = problem_for(w)
    rng = np.random.default_rng(23)
    x = w.q_cur + 3e-3 * rng.normal(size=w.q_cur.shape)  # every vertex moves
    y = O.predictor(P, w.q_cur, w.q_prev)
    cl = w.clamped.astype(bool)
    assert np.abs(x[cl] - y[cl]).max() > 1e-4
    with sim_for(w, prec, use_graph=0) as sim:
        g, grad = sim.energy_grad(x, y)
    g_ref = O.objective(P, x, y)
    assert abs(g - g_ref) <= (1e-11 if prec == FP64 else 2e-6) * abs(g_ref), (g, g_ref)
    assert rel(grad, O.gradient(P, x, y)) <= (1e-11 if prec == FP64 else 1e-5)
    assert np.all(grad[cl] == 0.0)


def test_energy_gradient_inverted_tets():
    """States with inverted elements exercise the Neo-Hookean continuation
    below J0 and the signed SVD (s3 < 0)."""
    w = W.lattice_workload((3, 3, 3), W.Material(W.NEOHOOKEAN, 1e5, 0.45), seed=5)
    P = problem_for(w)
    x = perturbed(w, 0.03, 7)
    F = O.deformation_gradients(P, x)
    assert np.sum(np.linalg.det(F) < 0) > 5
    y = w.q_cur
    for prec, tol in ((FP64, 1e-10), (FP32, 1e-5)):
        with sim_for(w, prec, use_graph=0) as sim:
            g, grad = sim.energy_grad(x, y)
        assert rel(grad, O.gradient(P, x, y)) <= tol
        assert abs(g - O.objective(P, x, y)) <= 10 * tol * abs(O.objective(P, x, y))


@pytest.mark.parametrize("kind", [W.COROTATED, W.POLY4])
def test_energy_gradient_other_materials(kind):
    w = W.lattice_workload((4, 3, 5), W.Material(kind, 2e5, 0.35), seed=9, v_range=0.3)
    P = problem_for(w)
    x = perturbed(w, 4e-3, 3)
    y = O.predictor(P, w.q_cur, w.q_prev)
    with sim_for(w, FP64, use_graph=0) as sim:
        g, grad = sim.energy_grad(x, y)
    assert rel(grad, O.gradient(P, x, y)) <= 1e-10
    assert abs(g - O.objective(P, x, y)) <= 1e-10 * abs(O.objective(P, x, y))


# ---------------------------------------------------------------- A0 solve and two-loop

# a lattice whose upper separators have backward rows long enough to be
# split into chunk items (rows of Q^T longer than 1024 entries)
LAT30 = W.lattice_workload((30, 30, 30), W.Material(W.NEOHOOKEAN, 5e5, 0.4), clamp_axis=2, seed=13, name="lat30")


# shapes of the sweeps (hqn_params.solve_*): block threads, work-item size
# and count, L2 prefetches (factor rows ahead; the dense block's matrix)
SHAPES = {"default": {}, "t512": dict(solve_threads=512),
          "small_items": dict(solve_item_kb=16, solve_items=2000, solve_prefetch=1),
          "big_items": dict(solve_item_kb=128, solve_items=152, solve_threads=512, solve_prefetch=4),
          "no_prefetch": dict(solve_prefetch=-1), "dense_prefetch": dict(solve_dense_prefetch=1, solve_dense_top=3),
          "dense_top1": dict(solve_dense_top=1), "dense_top3": dict(solve_dense_top=3, solve_prefetch=2),
          "no_dense_top": dict(solve_dense_top=-1),
          "leaf_items": dict(solve_leaf_kb=16, solve_leaf_threads=128, solve_threads=512)}


@pytest.mark.parametrize("w", WORKLOADS[:3] + [LAT30], ids=IDS[:3] + ["lat30"])
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("shape", sorted(SHAPES))
def test_solve_A0_parity(w, prec, shape):
    P = problem_for(w)
    rng = np.random.default_rng(4)
    q = rng.normal(size=(w.n_verts, 3))
    with sim_for(w, prec, use_graph=0, **SHAPES[shape]) as sim:
        info = sim.info()
        for k, v in SHAPES[shape].items():
            if k in ("solve_prefetch", "solve_dense_top") and v < 0:
                want = 0
            elif k == "solve_dense_top":
                want = min(v, info["n_levels"])
            else:
                want = v
            assert info[k] == want, (k, info[k])
        if SHAPES[shape].get("solve_dense_top", 0) > 0:
            assert info["dense_top_cols"] > 0
        elif SHAPES[shape].get("solve_dense_top", 0) < 0:
            assert info["dense_top_cols"] == 0
        r = sim.solve_A0(q)
    r_ref = O.solve_A(P, q)
    assert rel(r, r_ref) <= (1e-11 if prec == FP64 else 2e-5)
    assert np.all(r[w.clamped.astype(bool)] == 0.0)


@pytest.mark.parametrize("npairs", [0, 1, 3, 5])
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_direction_parity(npairs, prec):
    w = WORKLOADS[1]
    P = problem_for(w)
    rng = np.random.default_rng(10 + npairs)
    free = ~w.clamped.astype(bool)
    grad = rng.normal(size=(w.n_verts, 3)) * free[:, None]
    # t_i = A0 s_i + small noise keeps rho > 0 (a plausible curvature pair)
    pairs = []
    for _ in range(npairs):
        s = rng.normal(size=(w.n_verts, 3)) * free[:, None]
        t = np.zeros_like(s)
        t[free] = P.A @ s[free] + 0.01 * rng.normal(size=s[free].shape) * np.abs(P.A @ s[free]).mean()
        pairs.append((s, t, float(np.sum(s * t))))
    d_ref = O.lbfgs_direction(P, grad, pairs)
    with sim_for(w, prec, use_graph=0) as sim:
        d = sim.direction(grad, [p[0] for p in pairs], [p[1] for p in pairs])
    assert rel(d, d_ref) <= (1e-10 if prec == FP64 else 1e-4)


# ---------------------------------------------------------------- whole steps

# The step's own motion is the stricter yardstick of position errors:
# e_x' = ||x_GPU - x_oracle|| / ||x_oracle - q_l||.  FP64 agrees to rounding;
# FP32 rounds the state and every sweep to 24 bits, and the ten iterations
# of the (non-converged) step carry that rounding into x.
STEP_TOL = {FP64: 1e-8, FP32: 1e-3}


def rel_step(x, x_ref, q_l):
    return float(np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref - q_l))


def _step_parity(w, prec, use_graph, tol_x):
    P = problem_for(w)
    x_ref, st = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history)
    with sim_for(w, prec, use_graph=use_graph) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        rc, stats = sim.step(1, stats=True)
        qc, qp = sim.get_state()
    assert rc >= 0
    np.testing.assert_allclose(qp, w.q_cur, rtol=0, atol=1e-6 if prec == FP32 else 1e-14)
    ex = rel(qc, x_ref)
    assert ex <= tol_x, (ex, stats["trials"], st.trials)
    ex_step = rel_step(qc, x_ref, w.q_cur)
    assert ex_step <= STEP_TOL[prec], (ex_step, stats["trials"], st.trials)
    return stats, st, qc, x_ref


@pytest.mark.parametrize("w", WORKLOADS, ids=IDS)
def test_step_parity_fp64_eager(w):
    stats, st, qc, x_ref = _step_parity(w, FP64, 0, 1e-9)
    assert stats["trials"] == st.trials
    np.testing.assert_allclose(stats["g"], st.g, rtol=1e-9)


@pytest.mark.parametrize("w", WORKLOADS, ids=IDS)
def test_step_parity_fp32_eager(w):
    _step_parity(w, FP32, 0, 1e-4)


@pytest.mark.parametrize("w", WORKLOADS, ids=IDS)
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_step_parity_graph(w, prec):
    stats, st, qc, x_ref = _step_parity(w, prec, 1, 1e-9 if prec == FP64 else 1e-4)
    if prec == FP64:
        assert stats["trials"] == st.trials


def test_sweep_shapes_agree_bitwise():
    """The block's thread count and the L2 prefetch distance change neither
    the work items nor any row's summation order, so whole steps agree bit
    for bit; repeated solves on one handle (the chunk counters re-arm
    themselves) give the same result every time."""
    w = WORKLOADS[1]
    out = []
    for kw in ({}, dict(solve_threads=512), dict(solve_dense_prefetch=1), dict(solve_prefetch=6)):
        with sim_for(w, FP32, use_graph=1, **kw) as sim:
            sim.set_state(w.q_cur, w.q_prev)
            sim.step(3)
            out.append(sim.get_state()[0])
    for o in out[1:]:
        np.testing.assert_array_equal(out[0], o)
    rng = np.random.default_rng(12)
    q = rng.normal(size=(LAT30.n_verts, 3))
    with sim_for(LAT30, FP32, use_graph=0) as sim:
        r1 = sim.solve_A0(q)
        r2 = sim.solve_A0(q)
    np.testing.assert_array_equal(r1, r2)


STEP_SHAPES = {"small_items_t512": dict(solve_item_kb=16, solve_items=2000, solve_threads=512),
               "dense_top2": dict(solve_dense_top=2), "no_dense_top": dict(solve_dense_top=-1)}


@pytest.mark.parametrize("w", WORKLOADS, ids=IDS)
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("shape", sorted(STEP_SHAPES))
def test_step_parity_other_sweep_shapes(w, prec, shape):
    """Whole steps with other sweep shapes against the oracle, at the
    tolerances of the default shapes: small work items (other row splits,
    so other summation orders) with 512-thread blocks, the dense top block
    over the top two levels, and no dense top block at all (the default
    chooses it automatically)."""
    P = problem_for(w)
    x_ref, st = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history)
    with sim_for(w, prec, use_graph=1, **STEP_SHAPES[shape]) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        rc, stats = sim.step(1, stats=True)
        qc, _ = sim.get_state()
    assert rc >= 0
    assert rel(qc, x_ref) <= (1e-9 if prec == FP64 else 1e-4), rel(qc, x_ref)
    assert rel_step(qc, x_ref, w.q_cur) <= STEP_TOL[prec]
    if prec == FP64:
        assert stats["trials"] == st.trials


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_graph_equals_eager_bitwise(prec):
    w = WORKLOADS[2]
    out = []
    for g in (0, 1, 1):
        with sim_for(w, prec, use_graph=g) as sim:
            sim.set_state(w.q_cur, w.q_prev)
            sim.step(3)
            out.append(sim.get_state()[0])
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(out[1], out[2])


def test_trajectory_30_steps_fp64():
    """The FP64 form tracks the oracle over the bar's 30-step trajectory."""
    w = W.bar_4x4x16_fp64()
    P = problem_for(w)
    qc, qp = w.q_cur.copy(), w.q_prev.copy()
    with sim_for(w, FP64) as sim:
        sim.set_state(qc, qp)
        for k in range(30):
            x_ref, _ = O.solve_step(P, qc, qp, iters=10, m=5)
            qp, qc = qc, x_ref
            sim.step(1)
            gq, _ = sim.get_state()
            assert rel(gq, x_ref) <= 1e-8, k


@pytest.fixture(scope="module")
def lat30_solve_case():
    rng = np.random.default_rng(21)
    q = rng.normal(size=(LAT30.n_verts, 3))
    return q, O.solve_A(problem_for(LAT30), q)


@pytest.mark.parametrize("merge", [0, 1, 5, 0x55, 0x155], ids=lambda m: f"merge{m:#x}")
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("threads", [256, 512])
def test_solve_A0_merged_supernodes(lat30_solve_case, merge, prec, threads):
    """Supernodes that merge a separator with the separators under it (their
    update entries fed by up to four children) solve A0 r = q to the same
    tolerance as the plain dissection tree."""
    q, r_ref = lat30_solve_case
    with sim_for(LAT30, prec, use_graph=0, merge_depths=merge, solve_threads=threads) as sim:
        r = sim.solve_A0(q)
    assert rel(r, r_ref) <= (1e-11 if prec == FP64 else 2e-5)
    assert np.all(r[LAT30.clamped.astype(bool)] == 0.0)


def test_merged_supernodes_shorten_the_sweeps():
    """Each merged depth removes one level from the sweeps' chain; the
    default merges none; a mask with two adjacent depths is rejected."""
    from paper_1604_07378_gb300 import hqn
    levels = {}
    for merge in (0, 1, 5, 0x55):
        with sim_for(LAT30, FP32, merge_depths=merge) as sim:
            levels[merge] = sim.info()["n_levels"]
    assert levels[1] == levels[0] - 1 and levels[5] == levels[0] - 2
    assert levels[0x55] < levels[5]
    with sim_for(LAT30, FP32) as sim:
        assert sim.info()["n_levels"] == levels[0]
    with pytest.raises(hqn.HQNError) as e:
        sim_for(LAT30, FP32, merge_depths=3)
    assert e.value.code == hqn.HQN_ERR_ARG


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_positions_device_is_the_state(prec):
    """sim_positions_device: the device copy of q_l in the caller's vertex
    order equals the state sim_get_state downloads (FP64: bit for bit; FP32:
    rest + displacement added in float32, within one float32 rounding of
    the coordinates)."""
    w = WORKLOADS[1]
    with sim_for(w, prec) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        sim.step(2)
        x, _ = sim.get_state()
        t = sim.positions_device()
        p = t.double().cpu().numpy()
    assert p.shape == (w.n_verts, 4) and np.all(p[:, 3] == 0.0)
    if prec == FP64:
        np.testing.assert_array_equal(p[:, :3], x)
    else:
        assert np.abs(p[:, :3] - x).max() <= 2 ** -23 * np.abs(x).max() * 2


# ---------------------------------------------------------------- Alg. 1's trial cap, checkpoints

@pytest.mark.parametrize("use_graph", [0, 1], ids=["eager", "graph"])
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_line_search_exhaustion_status_and_state(prec, use_graph):
    """ls_max = 1 on the small twisted spline bar: the ninth iteration's
    alpha = 1 is rejected (the oracle's pins check it from Armijo's
    inequality), so the step ends at x_k with HQN_WARN_LS_EXHAUSTED -- on the
    device exactly as in the oracle."""
    from paper_1604_07378_gb300 import hqn
    w = W.spline_bar_80x40x40(scale=16)
    P = problem_for(w)
    x_ref, st = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history, ls_max=1)
    assert st.exhausted and len(st.trials) < w.iters
    with sim_for(w, prec, use_graph=use_graph, ls_max=1) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        rc, stats = sim.step(1, stats=True)
        qc, _ = sim.get_state()
    assert rc == hqn.HQN_WARN_LS_EXHAUSTED and stats["status"] == hqn.HQN_WARN_LS_EXHAUSTED
    assert stats["iters"] == len(st.trials), (stats["iters"], st.trials)
    assert rel(qc, x_ref) <= (1e-9 if prec == FP64 else 1e-4)
    assert rel_step(qc, x_ref, w.q_cur) <= STEP_TOL[prec]
    if prec == FP64:
        np.testing.assert_allclose(stats["g"], st.g, rtol=1e-9)


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_checkpoint_resume(prec):
    """The state (q_l, q_{l-1}) is the whole state between steps (the history
    is reset every step): 15 steps, sim_get_state, a new handle,
    sim_set_state and 15 more steps equal 30 straight steps.  FP32 holds the
    float32 displacement, which survives the float64 round trip X + u - X,
    so it is bit for bit; FP64's round trip rounds once in the sum."""
    w = WORKLOADS[2]
    with sim_for(w, prec) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        sim.step(30)
        straight, straight_prev = sim.get_state()
    with sim_for(w, prec) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        sim.step(15)
        qc, qp = sim.get_state()
    with sim_for(w, prec) as sim:
        sim.set_state(qc, qp)
        sim.step(15)
        resumed, resumed_prev = sim.get_state()
    if prec == FP32:
        np.testing.assert_array_equal(resumed, straight)
        np.testing.assert_array_equal(resumed_prev, straight_prev)
    else:
        assert rel(resumed, straight) <= 1e-12
        assert rel(resumed_prev, straight_prev) <= 1e-12


# ---------------------------------------------------------------- bounded device waits

@pytest.mark.parametrize("use_graph", [0, 1], ids=["eager", "graph"])
def test_sweep_wait_timeout_is_reported(use_graph):
    """Failure detection without a GPU fault: with fault_test = 1 the first
    forward level's blocks issue no copy, so each block's wait on its copy
    (bounded here to 2,000 polls) runs out with nothing in flight; the block
    flags it and leaves, and the step returns HQN_ERR_DEVICE_TIMEOUT instead
    of hanging.  The context stays usable: a new handle then steps as the
    oracle does."""
    from paper_1604_07378_gb300 import hqn
    w = WORKLOADS[1]
    # no dense top block: on this small mesh it would take the whole tree,
    # leaving no sweep level (and no copy wait) to make run out
    with sim_for(w, FP32, use_graph=use_graph, fault_test=1, wait_polls=2000, solve_dense_top=-1) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        with pytest.raises(hqn.HQNError) as e:
            sim.step(1)
        assert e.value.code == hqn.HQN_ERR_DEVICE_TIMEOUT
        with pytest.raises(hqn.HQNError) as e:
            sim.solve_A0(np.ones((w.n_verts, 3)))
        assert e.value.code == hqn.HQN_ERR_DEVICE_TIMEOUT
    P = problem_for(w)
    x_ref, _ = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history)
    with sim_for(w, FP32, use_graph=use_graph) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        assert sim.step(1) >= 0
        assert rel(sim.get_state()[0], x_ref) <= 1e-4


# ---------------------------------------------------------------- several materials in one mesh

TWO_MAT = W.two_material_bar((6, 4, 5), W.Material(W.NEOHOOKEAN, 2e5, 0.4, density=900.0),
                             W.Material(W.STVK, 8e5, 0.35, density=1300.0), seed=14, v_range=0.4,
                             name="two_material")


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_two_material_mesh_energy_solve_step(prec):
    """hqn_mesh.tet_material: each tet evaluated with its own material, its
    mass share and its weight in A0 from that material -- against the
    oracle: energy and gradient, A0^{-1}, one whole step (FP64 with the
    oracle's trial counts) and the Jacobi-PCG step (matrix-free A0 with the
    per-tet stiffness)."""
    w = TWO_MAT
    P = problem_for(w)
    assert len(P.mats) == 2
    y = O.predictor(P, w.q_cur, w.q_prev)
    x = perturbed(w, 4e-3, 2)
    q = np.random.default_rng(3).normal(size=(w.n_verts, 3))
    x_ref, st = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history)
    with sim_for(w, prec, use_graph=0) as sim:
        g, grad = sim.energy_grad(x, y)
        r = sim.solve_A0(q)
        sim.set_state(w.q_cur, w.q_prev)
        rc, stats = sim.step(1, stats=True)
        qc, _ = sim.get_state()
    tol = 1e-11 if prec == FP64 else 1e-5
    assert rel(grad, O.gradient(P, x, y)) <= tol
    assert abs(g - O.objective(P, x, y)) <= (1e-11 if prec == FP64 else 2e-6) * abs(O.objective(P, x, y))
    assert rel(r, O.solve_A(P, q)) <= (1e-11 if prec == FP64 else 2e-5)
    assert rc >= 0 and rel(qc, x_ref) <= (1e-9 if prec == FP64 else 1e-4)
    assert rel_step(qc, x_ref, w.q_cur) <= STEP_TOL[prec]
    if prec == FP64:
        assert stats["trials"] == st.trials
    x_pcg, _ = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history, pcg_iters=15)
    with sim_for(w, prec, a0_solver=1, pcg_iters=15) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        assert sim.step(1) >= 0
        assert rel(sim.get_state()[0], x_pcg) <= (1e-9 if prec == FP64 else 1e-4)


def test_two_material_mesh_in_a_batch_bitwise():
    """A batch mixing a two-material mesh with one-material meshes agrees bit
    for bit with single handles."""
    from paper_1604_07378_gb300 import hqn
    ws = [WORKLOADS[1], TWO_MAT, WORKLOADS[0]]
    with hqn.Batch(ws, precision=FP32) as b:
        for i, w in enumerate(ws):
            b.set_state(i, w.q_cur, w.q_prev)
        assert b.step(2)[0] >= 0
        got = [b.get_state(i)[0] for i in range(len(ws))]
    for i, w in enumerate(ws):
        with sim_for(w, FP32) as sim:
            sim.set_state(w.q_cur, w.q_prev)
            sim.step(2)
            np.testing.assert_array_equal(got[i], sim.get_state()[0])


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_energy_gradient_device_pointers(prec):
    """sim_energy_grad_device: the same g and grad g as sim_energy_grad (bit
    for bit: the same conversions, done on the device) and as the oracle, on
    caller-order float64 device arrays, clamped rows moved too."""
    torch = pytest.importorskip("torch")
    w = WORKLOADS[1]
    P = problem_for(w)
    rng = np.random.default_rng(31)
    x = w.q_cur + 3e-3 * rng.normal(size=w.q_cur.shape)
    y = O.predictor(P, w.q_cur, w.q_prev)
    stream = torch.cuda.current_stream()
    with sim_for(w, prec, use_graph=0, stream=stream.cuda_stream) as sim:
        g_h, grad_h = sim.energy_grad(x, y)
        xd = torch.tensor(x, dtype=torch.float64, device="cuda")
        yd = torch.tensor(y, dtype=torch.float64, device="cuda")
        for _ in range(2):
            g_d, grad_d = sim.energy_grad_device(xd, yd)
            grad_d = grad_d.cpu().numpy()
            assert g_d == g_h
            np.testing.assert_array_equal(grad_d, grad_h)
    assert abs(g_d - O.objective(P, x, y)) <= (1e-11 if prec == FP64 else 2e-6) * abs(O.objective(P, x, y))
    assert rel(grad_d, O.gradient(P, x, y)) <= (1e-11 if prec == FP64 else 1e-5)


def _inverted_at(w, x):
    X, T = w.rest_pos, w.tets
    Ds = np.stack([x[T[:, k]] - x[T[:, 0]] for k in (1, 2, 3)], axis=2)
    Dm = np.stack([X[T[:, k]] - X[T[:, 0]] for k in (1, 2, 3)], axis=2)
    return int((np.linalg.det(Ds) * np.linalg.det(Dm) < 0).sum())


# an 8^3 lattice whose every free vertex has its own velocity in [-1.5, 1.5]^3
# m/s: about a third of its 3,072 tets are inverted at the predictor y, and the
# line search backtracks (Neo-Hookean ~10 times per iteration, StVK in the
# first iterations)
TANGLED = [W.lattice_workload((8, 8, 8), W.Material(kind, 5e5, 0.4), clamp_axis=2, seed=31, v_range=1.5,
                              v_mode="iid", name=f"tangled8_{W.MATERIAL_NAMES[kind]}")
           for kind in (W.NEOHOOKEAN, W.STVK)]


@pytest.mark.parametrize("w", TANGLED, ids=[w.name for w in TANGLED])
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_tangled_lattice_step_parity(w, prec):
    """Inverted elements at scale: a whole step of a lattice tangled by
    per-vertex velocities (hundreds of inverted tets at y, rejected trials)
    against the oracle; FP64 with the oracle's trial counts."""
    P = problem_for(w)
    assert _inverted_at(w, O.predictor(P, w.q_cur, w.q_prev)) > 500
    stats, st, qc, x_ref = _step_parity(w, prec, 1, 1e-9 if prec == FP64 else 1e-4)
    assert sum(st.trials) > w.iters
    if prec == FP64:
        assert stats["trials"] == st.trials
