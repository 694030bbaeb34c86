"""The autotuner on the device: re-planning the sweeps of a live handle,
the tuning run itself on a small mesh, and sim_create applying the cache."""
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


W9 = W.lattice_workload((9, 8, 10), W.Material(W.NEOHOOKEAN, 5e5, 0.4), clamp_axis=2, seed=12, v_range=0.5,
                        v_mode="body", name="lat9x8x10")


@pytest.mark.parametrize("use_graph", [0, 1], ids=["eager", "graph"])
def test_replanned_sweeps_solve_and_step(use_graph):
    """sim_set_solve_shapes on a live handle: every shape of a sample of the
    grid solves A0 r = q as the oracle does, the step graph is rebuilt and
    a step after the last re-plan matches the oracle's."""
    from paper_1604_07378_gb300 import autotune, hqn
    w = W9
    P = problem_for(w)
    rng = np.random.default_rng(3)
    q = rng.normal(size=(w.n_verts, 3))
    r_ref = O.solve_A(P, q)
    x_ref, _ = O.solve_step(P, w.q_cur, w.q_prev, iters=w.iters, m=w.history)
    with hqn.Sim.from_workload(w, precision=FP32, use_graph=use_graph) as sim:
        for shape in autotune.SHAPE_GRID[::5] + (dict(solve_threads=128, solve_leaf_threads=512),):
            sim.set_solve_shapes(**shape)
            info = sim.info()
            for k in ("solve_threads", "solve_item_kb", "solve_items"):
                if shape.get(k):
                    assert info[k] == shape[k], (k, shape)
            if shape.get("solve_leaf_threads"):
                assert info["solve_leaf_threads"] == shape["solve_leaf_threads"]
            assert rel(sim.solve_A0(q), r_ref) <= 2e-5, shape
        with pytest.raises(hqn.HQNError):
            sim.set_solve_shapes(solve_threads=384)
        sim.set_state(w.q_cur, w.q_prev)
        assert sim.step(1) >= 0
        assert rel(sim.get_state()[0], x_ref) <= 1e-4


def test_tuning_writes_a_cache_that_sim_create_applies(tmp_path):
    """A small tuning run: the choice is no slower than the defaults on the
    steps it timed, its cache line is what the library looks up, and a handle
    created with tune_cache takes the tuned shapes and steps correctly."""
    from paper_1604_07378_gb300 import autotune, hqn
    w = W9
    cache = str(tmp_path / "cache.txt")
    grid = (dict(solve_dense_prefetch=1), dict(solve_item_kb=32, solve_items=800, solve_leaf_kb=16, solve_leaf_threads=128),
            dict(solve_threads=512, solve_item_kb=96, solve_items=152))
    res = autotune.tune_workload(w, leaf_sizes=(32, 64), dense_tops=(0, 2), grid=grid, reps=5, steps=3, cache=cache)
    assert res["step_ms"] <= res["default_step_ms"]
    key = autotune.mesh_key(w.rest_pos, w.tets, w.clamped)
    dev = autotune._device_name()
    hit = autotune.lookup(cache, dev, key, FP32)
    if res["leaf_size"] == 0 and "ls_batch" not in res:  # the defaults won: nothing written
        assert hit is None
        return
    assert hit["leaf_size"] == res["leaf_size"] and hit["solve_items"] == res["solve_items"]
    assert hit["solve_dense_top"] == res["solve_dense_top"]
    assert hit["ls_batch"] == res.get("ls_batch", 8)
    x_ref, _ = O.solve_step(problem_for(w), w.q_cur, w.q_prev, iters=w.iters, m=w.history)
    with hqn.Sim.from_workload(w, precision=FP32, tune_cache=cache) as sim:
        info = sim.info()
        # (zeros in the entry keep the library's defaults: 400 items of 64 KB)
        assert info["solve_items"] == (res["solve_items"] or 400)
        assert info["solve_item_kb"] == (res["solve_item_kb"] or 64)
        sim.set_state(w.q_cur, w.q_prev)
        assert sim.step(1) >= 0
        assert rel(sim.get_state()[0], x_ref) <= 1e-4
