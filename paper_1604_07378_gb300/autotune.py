"""The project's autotuner of the solver's launch shapes.

The speed of the A0^{-1} sweeps, the heaviest stage of a step, depends on
shapes the method leaves open: the nested-dissection leaf size (which sets
the factor's levels and fill), how many top levels of the tree are solved
by one dense block, the threads of a sweep block, the size and number of
the work items a level's rows are split into (the leaf level's on their
own), and what the levels prefetch into L2.  This module times them on the
current GPU, on the mesh itself:

1. for every (leaf size, dense top levels), one handle (one
   factorisation); on it every sweep shape of the grid is planned in turn
   (sim_set_solve_shapes re-plans the work items without refactorising)
   and one solve is timed with CUDA events on the device (sim_time_stage,
   best of three means);
2. the three fastest shapes of each handle, and the library's defaults,
   are timed as whole time steps (one CUDA graph each);
3. the line search's trials per pass (ls_batch, a creation parameter) is
   timed as whole steps with the fastest shapes, one handle per value;
4. the fastest is written to the cache file as one line, keyed by the
   device name, the precision and the mesh's hash (hqn_mesh_key).

sim_create reads the cache when hqn_params.tune_cache names it, so a tuned
mesh needs no timing afterwards.  The choice is never slower than the
defaults on the steps timed, since the defaults are among the candidates.
"""
from __future__ import annotations

import ctypes as C
import os
import time

import numpy as np

from . import hqn

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.txt")

LEAF_SIZES = (64, 128)
DENSE_TOPS = (-1, 2, 3)
LS_BATCHES = (4, 8, 16)  # trials per line-search pass (the library's default is 8)
SHAPE_KEYS = ("solve_threads", "solve_item_kb", "solve_items", "solve_prefetch", "solve_leaf_kb",
              "solve_leaf_threads", "solve_dense_prefetch")
# the re-plannable sweep shapes (hqn_params.solve_*; 0 = default)
SHAPE_GRID = tuple(dict(solve_threads=256, solve_item_kb=kb, solve_items=n, solve_dense_prefetch=dp,
                        solve_leaf_kb=lkb, solve_leaf_threads=lt)
                   for kb, n in ((64, 400), (48, 304), (96, 304))
                   for lkb, lt in ((0, 0), (24, 128), (32, 128), (48, 256))
                   for dp in (0, 1))
STEP_FINALISTS = 3  # the fastest solves of each handle, timed again as whole steps


def mesh_key(rest_pos, tets, clamped=None) -> int:
    """The library's hash of a mesh (hqn_mesh_key)."""
    X = np.ascontiguousarray(rest_pos, dtype=np.float64)
    T = np.ascontiguousarray(tets, dtype=np.int32)
    cl = None if clamped is None else np.ascontiguousarray(clamped, dtype=np.uint8)
    m = hqn.Mesh(X.shape[0], T.shape[0], X.ctypes.data_as(C.POINTER(C.c_double)),
                 T.ctypes.data_as(C.POINTER(C.c_int32)),
                 None if cl is None else cl.ctypes.data_as(C.POINTER(C.c_uint8)))
    return int(hqn.library().hqn_mesh_key(C.byref(m)))


def cache_line(device: str, precision: int, key: int, choice: dict, **extra) -> str:
    """One cache entry in the format hqn_tune_lookup reads."""
    fields = [f"device={device.replace(' ', '_')}", f"precision={int(precision)}", f"key={key:016x}",
              f"leaf_size={int(choice['leaf_size'])}", f"solve_dense_top={int(choice.get('solve_dense_top', 0))}"]
    fields += [f"{k}={int(choice.get(k, 0))}" for k in SHAPE_KEYS]
    if choice.get("ls_batch"):
        fields.append(f"ls_batch={int(choice['ls_batch'])}")
    fields += [f"{k}={v:.6g}" if isinstance(v, float) else f"{k}={v}" for k, v in extra.items()]
    return "hqn-tune 1 " + " ".join(fields)


def lookup(path: str, device: str, key: int, precision: int):
    """The entry the library would apply (a dict of the tuned fields), or None."""
    p = hqn.default_params()
    rc = hqn.library().hqn_tune_lookup(os.fsencode(path), device.encode(), key, precision, C.byref(p))
    if rc < 0:
        raise hqn.HQNError(rc, f"malformed autotuner cache {path}")
    if rc == 0:
        return None
    return {"leaf_size": p.leaf_size, "solve_dense_top": p.solve_dense_top, **{k: getattr(p, k) for k in SHAPE_KEYS},
            "ls_batch": p.ls_batch}


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _step_ms(sim, w, steps):
    sim.set_state(w.q_cur, w.q_prev)
    sim.step(2)
    sim.set_state(w.q_cur, w.q_prev)
    t0 = time.perf_counter()
    sim.step(steps)  # ends with a synchronising read of the control blocks
    return 1e3 * (time.perf_counter() - t0) / steps


def tune_workload(w, precision=hqn.FP32_MIXED, stream=None, leaf_sizes=LEAF_SIZES, dense_tops=DENSE_TOPS,
                  grid=SHAPE_GRID, reps=20, steps=10, cache: str | None = DEFAULT_CACHE,
                  ls_batches=LS_BATCHES, min_gain=0.01) -> dict:
    """Times the shapes on workload `w` (a workloads.Workload) and returns
    the choice with its measurements; appends it to `cache` unless None.
    A candidate replaces the current choice only when its step is faster by
    more than `min_gain` (a fraction: step times vary by about half a per
    cent from run to run)."""
    results = []
    for leaf in leaf_sizes:
        for top in dense_tops:
            try:
                sim = hqn.Sim.from_workload(w, precision=precision, stream=stream, leaf_size=leaf,
                                            solve_dense_top=top)
            except hqn.HQNError:
                continue  # e.g. a dense top block too large for this mesh
            with sim:
                sim.set_state(w.q_cur, w.q_prev)
                sim.step(1)
                timed = []
                for g, shape in enumerate(grid):
                    try:
                        sim.set_solve_shapes(**shape)
                    except hqn.HQNError:
                        continue  # items that do not fit a block's shared memory
                    t = min(sim.time_stage(hqn.STAGE_SOLVE, reps) for _ in range(3))
                    timed.append((t, g))
                if not timed:
                    continue
                # a shape may speed the solve and slow the rest of the step
                # (L2 traffic), so the whole step decides among the finalists
                finals = []
                for t_solve, g in sorted(timed)[:STEP_FINALISTS]:
                    sim.set_solve_shapes(**grid[g])
                    finals.append((_step_ms(sim, w, steps), t_solve, g))
                t_step, t_solve, g_best = min(finals)
                results.append({"leaf_size": leaf, "solve_dense_top": top, **grid[g_best], "solve_ms": t_solve,
                                "step_ms": t_step, "shapes_timed": len(timed)})
    with hqn.Sim.from_workload(w, precision=precision, stream=stream) as sim:
        info = sim.info()
        default = {"leaf_size": 0, "solve_dense_top": 0, **{k: 0 for k in SHAPE_KEYS},
                   "solve_ms": min(sim.time_stage(hqn.STAGE_SOLVE, reps) for _ in range(3)),
                   "step_ms": _step_ms(sim, w, steps), "levels": info["n_levels"]}
    best = min(results, key=lambda r: r["step_ms"]) if results else default
    choice = best if best["step_ms"] < default["step_ms"] * (1.0 - min_gain) else default
    tuned = choice is not default
    # trials per line-search pass, with the chosen shapes (a new handle each)
    base_lb = hqn.default_params().ls_batch
    shapes = {k: choice[k] for k in SHAPE_KEYS if choice.get(k)}
    lb_timed = []
    for lb in ls_batches:
        if lb == base_lb:
            continue
        with hqn.Sim.from_workload(w, precision=precision, stream=stream, leaf_size=choice["leaf_size"],
                                   solve_dense_top=choice["solve_dense_top"], ls_batch=lb, **shapes) as sim:
            lb_timed.append((_step_ms(sim, w, steps), lb))
    if lb_timed and min(lb_timed)[0] < choice["step_ms"] * (1.0 - min_gain):
        t, lb = min(lb_timed)
        choice = dict(choice, ls_batch=lb, step_ms=t)
        tuned = True
    out = dict(choice)
    out["ls_batch_step_ms"] = {str(lb): t for t, lb in lb_timed}
    out["default_step_ms"] = default["step_ms"]
    out["default_solve_ms"] = default["solve_ms"]
    out["candidates"] = results
    if cache and tuned:
        key = mesh_key(w.rest_pos, w.tets, w.clamped)
        line = cache_line(_device_name(), precision, key, choice, step_ms=float(choice["step_ms"]),
                          solve_ms=float(choice["solve_ms"]), workload=getattr(w, "name", "mesh"))
        with open(cache, "a") as f:
            f.write(line + "\n")
        out["cache_line"] = line
    return out
