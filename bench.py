#!/usr/bin/env python
"""Benchmark: implicit-Euler time steps per second of the quasi-Newton /
L-BFGS solver on the 40x40x40 Neo-Hookean tet lattice (384,000 tets,
68,921 vertices, E = 5e5, nu = 0.4, bottom face clamped, seeded initial
velocities U[-0.5, 0.5] m/s, 10 iterations, m = 5), FP32-mixed form, with the
FP64-plain GPU form and the FP64 CPU oracle beside it.

One "step" is one whole time step (predictor, 10 quasi-Newton iterations with
their line searches, commit) launched as one CUDA graph.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): one independent replica per rank (the single-mesh
path does not shard), value = all ranks' steps / slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-steps/s & tet grad-evals/s at 384k tets, FP32 vs FP64 GPU, pos err ≤1e-4"
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one cube40 FP32
# solve (default shapes: 7 forward levels, the dense top block, 7 backward
# levels), summed over its 15 launches in ncu captures of three launches each
# (232.79 MB read, 0.004 MB written); None when a sweep kernel changes until
# re-captured.
SOLVE_TRAFFIC_BYTES = 232_794_112
UNIT = "time-steps/s"
WORKLOAD = "cube40_neohookean"
# FP32 floating-point operations of the tet pass per tet (2 x FFMA + FADD +
# FMUL, from ncu's sass instruction counters on one k_tet launch of cube40,
# TET_EVAL: 46.85M FFMA, 55.68M FADD, 28.03M FMUL over 384,000 tets; MUFU
# operations not counted); None when the kernel changes until re-captured.
TET_FLOPS_PER_TET = 462.0
# per-tet-evaluation algorithmic bytes of the tet pass (idx 16 + Dm^-1 36 +
# V 4 B, plus the vertex data of x_k, d, x, grad, y and mass per vertex
# spread over the tets, 64 B x n / T); the solve's 2 nnz(L) x 4 B + 2 x 12 B
# x n_f; the two-loop's (96 m + 48) B per vertex per iteration
TET_BYTES = 56.0
VERT_BYTES = 64.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- oracle (CPU)

def host_description():
    """The host cores the CPU timings ran on: logical CPUs, those this
    process may use, and the CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu model")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"nproc": os.cpu_count(), "usable": usable, "model": model or "unknown"}


def oracle_child(args):
    """Runs in a child process (its thread count fixed by the environment
    before numpy loads): whole FP64 oracle steps of cube40 (Alg. 1 with
    Alg. 2, 10 iterations, m = 5, the workload's own state carried from step
    to step), as many as fit in the budget (at least one); the oracle's A0
    factorisation is set-up, not timed.  Prints one JSON line."""
    from oracle import hqn_oracle as O
    from paper_1604_07378_gb300 import workloads as W
    w = W.cube40(W.NEOHOOKEAN)
    P = O.problem_from_workload(w)
    O.solve_A(P, np.zeros_like(w.q_cur))  # factorisation
    qc, qp = w.q_cur.copy(), w.q_prev.copy()
    steps = trials = iters = 0
    wall0, cpu0 = time.perf_counter(), time.process_time()
    while steps < args.oracle_max_steps:
        x, st = O.solve_step(P, qc, qp, iters=w.iters, m=w.history)
        qp, qc = qc, x
        steps += 1
        trials += sum(st.trials)
        iters += len(st.trials)
        el = time.perf_counter() - wall0
        if el + el / steps > args.oracle_budget:
            break
    wall = time.perf_counter() - wall0
    cpu = time.process_time() - cpu0
    print(json.dumps({"steps": steps, "wall_s": wall, "cpu_s": cpu, "trials": trials, "iters": iters,
                      "tets": w.n_tets}), flush=True)


def oracle_steps(budget_s, threads, max_steps=1000):
    """Whole oracle steps of cube40 timed in a child process allowed
    `threads` threads (OpenMP / BLAS); returns the child's record with the
    time-steps/s and the cores it kept busy (CPU time over wall time)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-child", "--oracle-budget", str(budget_s),
           "--oracle-max-steps", str(max_steps)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=budget_s * 6 + 600)
    if r.returncode != 0:
        raise RuntimeError("oracle child failed:\n" + r.stderr[-2000:])
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    rec["threads_allowed"] = threads
    rec["cores"] = rec["cpu_s"] / rec["wall_s"]
    rec["steps_per_s"] = rec["steps"] / rec["wall_s"]
    rec["tet_grad_evals_per_s"] = rec["tets"] * (rec["trials"] + rec["steps"]) / rec["wall_s"]
    rec["ls_trials_per_iter"] = rec["trials"] / max(rec["iters"], 1)
    return rec


# ---------------------------------------------------------------------------- GPU arm

def solve_shapes(args):
    """hqn_params.solve_* from the command line (0 = the library default)."""
    return dict(solve_threads=args.solve_threads, solve_item_kb=args.solve_item_kb,
                solve_items=args.solve_items, solve_prefetch=args.solve_prefetch)


def max_over_ranks(x, dist, device=None):
    """The maximum of x over the ranks of the process group (x itself without
    one); every rank returns it.  The ranks first meet at a barrier."""
    if not dist:
        return float(x)
    import torch

    dist.barrier()
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, ms):
    """Whole-job time-steps per second: every rank advances its own replica
    `steps` steps, timed by the slowest rank (ms)."""
    return world * steps / (ms / 1e3)


def run_ours(args, rank, world, dist):
    import torch

    from paper_1604_07378_gb300 import hqn
    from paper_1604_07378_gb300 import workloads as W

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    from paper_1604_07378_gb300 import autotune
    w = W.cube40(W.NEOHOOKEAN)
    T = w.n_tets
    graph = 0 if args.no_graph else 1
    # the autotuner's choice for this mesh and GPU, if its cache has one and
    # no shape is forced on the command line
    forced = args.leaf_size or any(solve_shapes(args).values())
    tune_cache = None if forced or args.no_tune_cache else autotune.DEFAULT_CACHE
    tuned = None
    if tune_cache and os.path.exists(tune_cache):
        tuned = autotune.lookup(tune_cache, torch.cuda.get_device_name(dev), autotune.mesh_key(w.rest_pos, w.tets,
                                w.clamped), hqn.FP32_MIXED)
    sim = hqn.Sim.from_workload(w, precision=hqn.FP32_MIXED, stream=stream.cuda_stream, use_graph=graph,
                                leaf_size=args.leaf_size, tune_cache=tune_cache, **solve_shapes(args))
    info = sim.info()
    sim.set_state(w.q_cur, w.q_prev)
    sim.step(args.warmup)
    sim.set_state(w.q_cur, w.q_prev)

    # ---- timed region: K steps, one graph launch each
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev.index)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc, stats = sim.step(args.steps, stats=True)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    ms_step = ms / args.steps
    trials = stats["trials_total"] / args.steps
    iters = stats["iters_total"] / args.steps
    # energy evaluations per step: x_1 = y plus every line-search trial
    tet_evals_step = T * (stats["trials_total"] + args.steps) / args.steps
    value = job_throughput(world, args.steps, ms)

    # ---- per-stage device times (CUDA events on the handle's stream)
    stage_ms = {name: sim.time_stage(code, 20) for name, code in (
        ("tet", hqn.STAGE_TET), ("gather", hqn.STAGE_GATHER), ("solve", hqn.STAGE_SOLVE),
        ("ls_pass", hqn.STAGE_LS_PASS), ("two_loop_with_solve", hqn.STAGE_TWO_LOOP))}
    # line-search passes: the fused first trial (a tet pass with the gradient)
    # of every iteration plus the multi-trial passes after a rejection
    passes = stats["ls_passes_total"] / args.steps
    per_step = {"tet": stage_ms["tet"] * (iters + 1), "solve": stage_ms["solve"] * iters,
                "gather": stage_ms["gather"] * (iters + 1),
                "ls_pass": stage_ms["ls_pass"] * max(passes - iters, 0.0),
                "two_loop": max(stage_ms["two_loop_with_solve"] - stage_ms["solve"], 0.0) * iters}
    dominant = max(per_step, key=per_step.get)

    # ---- end to end through the C ABI with host buffers
    lib = hqn.library()
    import ctypes as C
    qc = np.ascontiguousarray(w.q_cur)
    qp = np.ascontiguousarray(w.q_prev)
    out = np.empty_like(qc)
    dp = C.POINTER(C.c_double)
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        lib.sim_set_state(sim._h, qc.ctypes.data_as(dp), qp.ctypes.data_as(dp))
        lib.sim_step(sim._h, 1, None)
        lib.sim_get_state(sim._h, out.ctypes.data_as(dp), None)
        qp, qc = qc, out.copy()
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_wall = time.perf_counter() - t0
    e2e_ms = max_over_ranks(max(f0.elapsed_time(f1), e2e_wall * 1e3), dist, dev)
    n = w.n_verts
    vbytes = 16  # FP32 vertex record
    h2d = 2 * n * vbytes
    d2h = n * vbytes + 1024  # state + control block (line-search statistics)

    # ---- FP64-plain GPU form beside it, and the accuracy of the FP32 form against it
    sim64 = hqn.Sim.from_workload(w, precision=hqn.FP64_PLAIN, stream=stream.cuda_stream, use_graph=graph,
                                  leaf_size=args.leaf_size, **solve_shapes(args))
    sim64.set_state(w.q_cur, w.q_prev)
    sim64.step(1)
    x64, _ = sim64.get_state()
    sim.set_state(w.q_cur, w.q_prev)
    sim.step(1)
    x32, _ = sim.get_state()
    ex = float(np.linalg.norm(x32 - x64) / np.linalg.norm(x64))
    ex_step = float(np.linalg.norm(x32 - x64) / np.linalg.norm(x64 - w.q_cur))
    k64 = max(2, min(args.steps, 4))
    sim64.set_state(w.q_cur, w.q_prev)
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    _, st64 = sim64.step(k64, stats=True)
    g1.record(stream)
    torch.cuda.synchronize()
    ms64 = g0.elapsed_time(g1) / k64
    tev64 = T * (st64["trials_total"] + k64) / k64
    sim64.close()

    # ---- roofline of the dominant kernel
    peaks, src = _peaks()
    fl = None
    if dominant == "solve":
        bytes_launch = 2 * info["factor_nnz"] * 4 + 2 * 12 * info["n_free"]
        achieved = bytes_launch / (stage_ms["solve"] * 1e-3) / 1e9
        roof = {"bound": "hbm",
                "kernel": "A0^-1 solve: forward sweep levels, dense top block, backward sweep levels "
                          "(k_fwd, k_dense, k_bwd), one solve",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                # the capture holds for the default tree and schedule only
                "traffic": SOLVE_TRAFFIC_BYTES if args.leaf_size == 0 and tuned is None else None,
                "algorithmic_bytes_per_launch": bytes_launch}
    else:
        # the tet pass (energy + corner gradients): idx 16 + Dm^-1 36 + V 4 B
        # and 4 corner gradients of 16 B per tet, x_k and d of every vertex
        dominant = "tet"
        bytes_launch = T * (56 + 64) + n * 32
        achieved = bytes_launch / (stage_ms["tet"] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                "algorithmic_bytes_per_launch": bytes_launch}
    roof["peak_source"] = f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src

    # ---- the whole step against the HBM roofline: algorithmic bytes of every
    # stage of a step (tet passes, solves, two-loop) over the step's time
    nf = info["n_free"]
    m = w.history
    solve_bytes = 2 * info["factor_nnz"] * 4 + 2 * 12 * nf
    step_bytes = (tet_evals_step * (TET_BYTES + VERT_BYTES * n / T) + iters * solve_bytes
                  + iters * (96 * m + 48) * n)
    roof_step = {"bound": "hbm", "algorithmic_bytes_per_step": step_bytes,
                 "achieved": step_bytes / (ms_step * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": step_bytes / (ms_step * 1e-3) / 1e9 / peaks["hbm_gbs"], "peak_source": roof["peak_source"]}

    # ---- the FP32 pipe: measured FMA-chain peak and the tet pass against it
    clk_peak = ClockSampler(dev.index)
    clk_peak.start()
    fp32_peak = hqn.measure_peak(hqn.FP32_MIXED)
    fp64_peak = hqn.measure_peak(hqn.FP64_PLAIN)
    peak_clocks = clk_peak.stop()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fma = {"fp32_tflops_measured": fp32_peak / 1e12, "fp64_tflops_measured": fp64_peak / 1e12,
           "sm_mhz_during": peak_clocks.get("sm_mhz"),
           "fp32_tflops_nominal_at_that_clock": (sms * 128 * 2 * peak_clocks["sm_mhz"] * 1e6 / 1e12
                                                 if peak_clocks.get("sm_mhz") else None)}
    tet_flops = None
    if TET_FLOPS_PER_TET:
        achieved = TET_FLOPS_PER_TET * T / (stage_ms["tet"] * 1e-3)
        tet_flops = {"bound": "fp32", "flops_per_tet": TET_FLOPS_PER_TET, "achieved_tflops": achieved / 1e12,
                     "peak_tflops": fp32_peak / 1e12, "frac": achieved / fp32_peak,
                     "hbm_frac": T * (TET_BYTES + 64.0) / (stage_ms["tet"] * 1e-3) / 1e9 / peaks["hbm_gbs"]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (f64 energy sums, Armijo test, inner products)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": "40x40x40 Kuhn cubes", "tets": T,
                   "vertices": n, "material": "Neo-Hookean E=5e5 nu=0.4", "iters": w.iters,
                   "history_m": w.history, "h": w.h, "parallelism": f"replicas{world}",
                   "initial_velocity": "one seeded body velocity, U[-0.5, 0.5]^3 m/s",
                   "chained_sweeps": bool(info.get("chained_sweeps", 0)),
                   "solve_shapes": {k: info[k] for k in ("n_levels", "solve_dense_top", "dense_top_cols",
                                                         "solve_threads", "solve_item_kb", "solve_items",
                                                         "solve_leaf_kb", "solve_leaf_threads",
                                                         "solve_prefetch")},
                   "tuned": tuned is not None,
                   "l2": "working set %.0f MB > 129 MB L2 (factor alone %.0f MB)" % (
                       info["device_bytes"] / 1e6, info["factor_entries"] * 4 / 1e6)},
        "tet_grad_evals_per_s": world * tet_evals_step * args.steps / (ms / 1e3),
        "ls_trials_per_iter": trials / max(iters, 1),
        "fp64_plain": {"value": 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64,
                       "tet_grad_evals_per_s": tev64 * 1e3 / ms64, "steps": k64},
        "pos_err_fp32_vs_fp64_gpu": ex,
        "pos_err_step_fp32_vs_fp64_gpu": ex_step,
        "stage_ms_per_launch": stage_ms, "stage_ms_per_step": per_step,
        "roofline": roof, "roofline_step": roof_step, "fma_peak": fma, "tet_flop_roofline": tet_flops,
        "clocks": clocks,
        "e2e": {"value": job_throughput(world, e2e_steps, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": None,
        "status": rc,
    }
    # kernels per step: start (predictor, inertia, tet, gather) + commit; per
    # iteration: q, the sweeps (2 per tree level), t^T r0 products (m > 0),
    # direction final, tet gradient (returns at once after an accepted first
    # trial), gather; plus every line-search pass (fused first trial included)
    m = w.history
    per_iter = 1 + 2 * info["n_levels"] + (1 if m > 0 else 0) + 1 + 2
    launches = args.steps * 5 + stats["iters_total"] * per_iter + stats["ls_passes_total"]
    line["gpu_launches"] = launches
    if not args.no_batch:
        line["batched"] = run_batched(args, stream, rank, world, dist)
    if not args.no_collisions:
        line["collisions"] = run_collisions(args, stream)
    if not args.no_pcg:
        line["a0_pcg"] = run_pcg(args, stream, x32)
    if not args.no_convergence:
        line["convergence"] = run_convergence(args, stream)
    if not args.no_configs:
        line["other_configs"] = run_other_configs(args, stream)
        line["other_configs"].update(run_small_configs(args, stream))
    if rank == 0 and not args.no_cpu_baseline:
        host = host_description()
        one = oracle_steps(args.cpu_budget, 1, max_steps=2)
        line["cpu_baseline"] = {
            "value": one["steps_per_s"], "unit": UNIT, "cores": round(one["cores"], 2), "kind": "oracle",
            "sample": f"{one['steps']} whole FP64 oracle step(s) of the same workload (10 iterations, m = 5, "
                      f"{one['trials']} line-search trials), {one['wall_s']:.1f} s wall, one thread allowed",
            "tet_grad_evals_per_s": one["tet_grad_evals_per_s"], "host": host}
        if not args.no_threaded_oracle:
            thr = oracle_steps(args.cpu_budget, host["usable"], max_steps=2)
            line["cpu_baseline"]["threaded"] = {
                "value": thr["steps_per_s"], "threads_allowed": thr["threads_allowed"],
                "cores_busy": round(thr["cores"], 2), "steps": thr["steps"], "wall_s": thr["wall_s"],
                "note": "the oracle is numpy/scipy: OpenMP/BLAS threads allowed, cores_busy measured"}
    sim.close()
    return line


def run_pcg(args, stream, x_direct):
    """The iterative alternative to the factorised A0^{-1} (the paper's
    comparison with iterative solvers): cube40, FP32-mixed, Jacobi-PCG with
    5 and 15 iterations in every L-BFGS direction; time-steps/s, the solve's
    time and the position difference from the direct-solve step."""
    import torch

    from paper_1604_07378_gb300 import hqn
    from paper_1604_07378_gb300 import workloads as W

    w = W.cube40(W.NEOHOOKEAN)
    out = {"workload": WORKLOAD}
    for iters in (5, 15):
        sim = hqn.Sim.from_workload(w, precision=hqn.FP32_MIXED, stream=stream.cuda_stream,
                                    a0_solver=1, pcg_iters=iters)
        sim.set_state(w.q_cur, w.q_prev)
        sim.step(1)
        x, _ = sim.get_state()
        ex = float(np.linalg.norm(x - x_direct) / np.linalg.norm(x_direct))
        sim.set_state(w.q_cur, w.q_prev)
        sim.step(2)
        steps = 20
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, st = sim.step(steps, stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        solve_ms = sim.time_stage(hqn.STAGE_SOLVE, 10)
        sim.close()
        out[f"pcg{iters}"] = {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "solve_ms": solve_ms, "status": rc,
                              "ls_trials_per_iter": st["trials_total"] / max(1, st["iters_total"]),
                              "pos_err_vs_direct_one_step": ex}
    return out


def run_other_configs(args, stream):
    """The other single-mesh workloads, FP32-mixed, one graph per step:
    the twisting spline bar (80x40x40, 768,000 tets, 10 iterations, m = 5)
    and the large bar (48x48x192, 2,654,208 tets, 20 iterations, m = 8) with
    one FP64-plain step beside it for the position difference."""
    import torch

    from paper_1604_07378_gb300 import hqn
    from paper_1604_07378_gb300 import workloads as W

    out = {}
    for key, w, steps in (("splinebar80x40x40", W.spline_bar_80x40x40(), 10),
                          ("largebar48x48x192", W.large_48x48x192(), 5)):
        t0 = time.perf_counter()
        sim = hqn.Sim.from_workload(w, precision=hqn.FP32_MIXED, stream=stream.cuda_stream,
                                    leaf_size=args.leaf_size, **solve_shapes(args))
        create_s = time.perf_counter() - t0
        sim.set_state(w.q_cur, w.q_prev)
        sim.step(1)
        x32, _ = sim.get_state()
        sim.set_state(w.q_cur, w.q_prev)
        sim.step(2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, st = sim.step(steps, stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        solve_ms = sim.time_stage(hqn.STAGE_SOLVE, 5)
        info = sim.info()
        sim.close()
        entry = {"tets": w.n_tets, "vertices": w.n_verts, "iters": w.iters, "history_m": w.history,
                 "steps_per_s": 1e3 / ms, "ms_per_step": ms, "steps": steps, "status": rc,
                 "tet_grad_evals_per_s": w.n_tets * (st["trials_total"] + steps) / steps * 1e3 / ms,
                 "ls_trials_per_iter": st["trials_total"] / max(1, st["iters_total"]),
                 "solve_ms": solve_ms, "factor_nnz": info["factor_nnz"], "create_s": create_s}
        if key.startswith("large"):
            sim64 = hqn.Sim.from_workload(w, precision=hqn.FP64_PLAIN, stream=stream.cuda_stream)
            sim64.set_state(w.q_cur, w.q_prev)
            torch.cuda.synchronize()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            sim64.step(1)
            g1.record(stream)
            torch.cuda.synchronize()
            x64, _ = sim64.get_state()
            sim64.close()
            entry["fp64_plain_steps_per_s"] = 1e3 / g0.elapsed_time(g1)
            entry["pos_err_fp32_vs_fp64_gpu"] = float(np.linalg.norm(x32 - x64) / np.linalg.norm(x64))
        out[key] = entry
    return out


def _timed_steps(sim, stream, steps):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc, st = sim.step(steps, stats=True)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, rc, st


def run_small_configs(args, stream):
    """The configurations beside the headline: the 4x4x16 bar in the plain
    FP64 form over its 30 steps; cube40 with St. Venant-Kirchhoff; cube40
    with the per-vertex iid initial velocities (a tangled mesh whose line
    search backtracks), over its first 20 steps."""
    from paper_1604_07378_gb300 import hqn
    from paper_1604_07378_gb300 import workloads as W

    out = {}
    w = W.bar_4x4x16_fp64()
    with hqn.Sim.from_workload(w, precision=hqn.FP64_PLAIN, stream=stream.cuda_stream) as sim:
        sim.set_state(w.q_cur, w.q_prev)
        sim.step(2)
        sim.set_state(w.q_cur, w.q_prev)
        ms, rc, st = _timed_steps(sim, stream, 30)
    out["bar4x4x16_fp64_plain"] = {"tets": w.n_tets, "vertices": w.n_verts, "precision": "f64", "steps": 30,
                                   "steps_per_s": 1e3 / ms, "ms_per_step": ms, "status": rc,
                                   "ls_trials_per_iter": st["trials_total"] / max(1, st["iters_total"])}
    for key, wl in (("cube40_stvk", W.cube40(W.STVK)),
                    ("cube40_neohookean_iid_velocity", W.cube40(W.NEOHOOKEAN, v_mode="iid"))):
        with hqn.Sim.from_workload(wl, precision=hqn.FP32_MIXED, stream=stream.cuda_stream) as sim:
            sim.set_state(wl.q_cur, wl.q_prev)
            sim.step(2)
            sim.set_state(wl.q_cur, wl.q_prev)
            ms, rc, st = _timed_steps(sim, stream, 20)
        out[key] = {"tets": wl.n_tets, "steps": 20, "steps_per_s": 1e3 / ms, "ms_per_step": ms, "status": rc,
                    "tet_grad_evals_per_s": wl.n_tets * (st["trials_total"] + 20) / 20 * 1e3 / ms,
                    "ls_trials_per_iter": st["trials_total"] / max(1, st["iters_total"]),
                    "initial_velocity": wl.meta.get("v_mode", "body")}
    return out


def run_convergence(args, stream):
    """Eq. RelativeError of one frame of the twisting spline bar (80x40x40 at
    half resolution, 96,000 tets, FP64): (g(x_k) - g(x*)) / (g(x_0) - g(x*))
    after 10, 30 and 60 iterations for projective dynamics (m = 0), L-BFGS
    with m = 2, 5, 8, 16, 100 and the Chebyshev direction (S = 10, rho
    estimated from a projective-dynamics run, and rho = 0.99),
    with the time per iteration; x* is a 500-iteration L-BFGS (m = 16) run
    (the paper's Newton reference is not built on the GPU)."""
    import torch

    from paper_1604_07378_gb300 import hqn
    from paper_1604_07378_gb300 import workloads as W

    w = W.spline_bar_80x40x40(scale=2)

    def run(iters, **kw):
        sim = hqn.Sim.from_workload(w, precision=hqn.FP64_PLAIN, stream=stream.cuda_stream, iters=iters, **kw)
        sim.set_state(w.q_cur, w.q_prev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = sim.step(1, stats=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sim.close()
        return st, dt

    st_star, _ = run(500, history_m=16)
    gs = st_star["g"]  # the step ends early once the line search can no longer decrease g
    g_star = min(gs)
    out = {"workload": "splinebar40x20x20_twist90", "tets": w.n_tets, "precision": "f64",
           "g_star_reference": "min g of an L-BFGS (m = 16) step of up to 500 iterations",
           "g_star_iterations": len(gs), "g_star_status": st_star["status"], "methods": {}}
    from paper_1604_07378_gb300 import chebyshev
    # rho of Alg. 3 estimated from a projective-dynamics run on the same frame
    st_pd, _ = run(150, history_m=0)
    rho_est = chebyshev.estimate_rho([st_pd["g0"]] + st_pd["g"])
    out["cheb_rho_estimated"] = rho_est
    out["cheb_rho_estimate"] = "sqrt of the median ratio of successive g decrements over the last 12 " \
                               "iterations of a 150-iteration projective-dynamics (m = 0) step"
    for name, kw in (("pd_m0", dict(history_m=0)), ("lbfgs_m2", dict(history_m=2)),
                     ("lbfgs_m5", dict(history_m=5)), ("lbfgs_m8", dict(history_m=8)),
                     ("lbfgs_m16", dict(history_m=16)), ("lbfgs_m100", dict(history_m=100)),
                     ("chebyshev_S10_rho_estimated", dict(direction=1, cheb_S=10, cheb_rho=rho_est)),
                     ("chebyshev_S10_rho0.99", dict(direction=1, cheb_S=10, cheb_rho=0.99))):
        st, dt = run(60, **kw)
        g = st["g"][:60]
        rel_err = {str(k): (g[k - 1] - g_star) / (st["g0"] - g_star) for k in (10, 30, 60)}
        out["methods"][name] = {"relative_error": rel_err, "ms_per_iteration": 1e3 * dt / 60,
                                "ls_trials_per_iter": st["trials_total"] / max(1, st["iters_total"])}
    return out


def run_collisions(args, stream):
    """Collision terms (Sec. 4.3): an unclamped 40^3 Neo-Hookean cube
    (384,000 tets) falling at 2 m/s onto a ground plane and a sphere, timed
    over the impact; FP32-mixed, one graph per step."""
    import torch

    from paper_1604_07378_gb300 import hqn
    from paper_1604_07378_gb300 import workloads as W

    w = W.collision_drop(40, drop=0.01, speed=2.0)
    sim = hqn.Sim.from_workload(w, precision=hqn.FP32_MIXED, stream=stream.cuda_stream,
                                leaf_size=args.leaf_size, **solve_shapes(args))
    sim.set_state(w.q_cur, w.q_prev)
    sim.step(2)  # warm-up: the fall before the impact
    steps = 20
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    rc, st = sim.step(steps, stats=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    x, _ = sim.get_state()
    sim.close()
    return {"workload": "drop40_plane_sphere", "tets": w.n_tets, "colliders": ["plane", "sphere"],
            "contact_scale": w.contact_scale, "steps_per_s": 1e3 / ms, "ms_per_step": ms, "steps": steps,
            "status": rc, "ls_trials_per_iter": st["trials_total"] / max(1, st["iters_total"]),
            "min_height_m": float(x[:, 2].min())}


def shard_batch(items, rank, world):
    """The simulations rank `rank` of `world` advances: a round-robin share,
    so every rank gets the same mix of sizes and materials.  Independent
    simulations need no data exchange between ranks."""
    return list(items[rank::world])


def run_batched(args, stream, rank=0, world=1, dist=None):
    """The batched form: 512 independent simulations (lattices of random
    dims 4-24 per axis, Neo-Hookean / StVK / spline materials, E log-uniform
    1e4-1e6, nu U[0.3, 0.48]) advanced together, one launch per kernel stage,
    one CUDA graph per step; FP32-mixed with the FP64-plain batch beside it.
    With several ranks the 512 simulations are sharded across them (no
    collective on the data path); simulation-steps/s counts all ranks'
    simulations over the slowest rank's time."""
    import torch

    from paper_1604_07378_gb300 import hqn
    from paper_1604_07378_gb300 import workloads as W

    all_ws = W.batch_512()
    ws = shard_batch(all_ws, rank, world)
    T = sum(w.n_tets for w in ws)
    out = {"workload": "batch512_lattices_4to24", "sims": len(all_ws), "sims_per_rank": len(ws), "ranks": world,
           "tets_total": sum(w.n_tets for w in all_ws), "vertices_total": sum(w.n_verts for w in all_ws)}
    for prec, key, steps in ((hqn.FP32_MIXED, "fp32_mixed", args.batch_steps),
                             (hqn.FP64_PLAIN, "fp64_plain", max(2, args.batch_steps // 4))):
        t0 = time.perf_counter()
        b = hqn.Batch(ws, precision=prec, stream=stream.cuda_stream, **solve_shapes(args))
        create_s = time.perf_counter() - t0
        for i, w in enumerate(ws):
            b.set_state(i, w.q_cur, w.q_prev)
        b.step(args.warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        rc, tot = b.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dist, torch.device("cuda", torch.cuda.current_device())) / steps
        info = b.info()
        solve_ms = b.time_stage(hqn.STAGE_SOLVE, 10)
        # the step's stages over the whole batch, one launch each (CUDA events)
        stages = {name: b.time_stage(st, 10) for name, st in
                  (("tet", hqn.STAGE_TET), ("gather", hqn.STAGE_GATHER), ("solve", hqn.STAGE_SOLVE),
                   ("two_loop_with_solve", hqn.STAGE_TWO_LOOP))}
        b.close()
        # tet evaluations per batch step: every simulation's start-of-step pass
        # and line-search passes (ls_passes_total is summed over the batch;
        # the simulations' sizes weight them equally here)
        evals = T * (tot["ls_passes_total"] / (steps * len(ws)) + 1)
        solve_bytes = 2 * info["factor_nnz"] * (4 if prec == hqn.FP32_MIXED else 8)
        peaks, _ = _peaks()
        out[key] = {"batch_steps_per_s": 1e3 / ms, "sim_steps_per_s": len(all_ws) * 1e3 / ms, "ms_per_step": ms,
                    "tet_grad_evals_per_s": evals * 1e3 / ms, "steps": steps, "status": rc,
                    "ls_trials_per_iter": tot["trials_total"] / max(tot["iters_total"], 1),
                    "create_s": create_s, "device_bytes": info["device_bytes"],
                    "solve_ms": solve_ms, "solve_hbm_frac_of_measured": solve_bytes / (solve_ms * 1e-3) / 1e9
                    / peaks["hbm_gbs"], "stage_ms_per_launch": stages,
                    # simulation-iterations that ran, of sims x iterations x steps (the rest
                    # ended early and idled in the batch's launches)
                    "sim_iterations_active_fraction": tot["iters_total"] / (len(ws) * ws[0].iters * steps)}
    return out


def run_reference(args, rank):
    """The reference arm: the FP64 CPU oracle itself (there is no reference
    implementation; the reference is the paper), rank 0 only.  Whole oracle
    time steps of the same workload, as many as fit in --ref-budget seconds
    (at least one): `steps` reports the steps actually timed, not K.  The
    oracle's A0 factorisation is set-up, not timed."""
    from paper_1604_07378_gb300 import workloads as W
    w = W.cube40(W.NEOHOOKEAN)
    host = host_description()
    rec = oracle_steps(args.ref_budget, host["usable"], max_steps=max(1, args.steps))
    value = rec["steps_per_s"]
    desc = (f"{rec['steps']} whole FP64 oracle step(s) of cube40 (10 iterations, m = 5, "
            f"{rec['trials']} line-search trials) in {rec['wall_s']:.1f} s; {args.steps} requested, "
            f"bounded by a {args.ref_budget:.0f} s budget")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": rec["steps"], "requested_steps": args.steps, "warmup": 0, "ms_per_step": 1e3 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "tets": w.n_tets, "vertices": w.n_verts,
                                            "iters": w.iters, "history_m": w.history},
            "tet_grad_evals_per_s": rec["tet_grad_evals_per_s"], "ls_trials_per_iter": rec["ls_trials_per_iter"],
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": round(rec["cores"], 2), "kind": "oracle",
                             "sample": desc, "threads_allowed": rec["threads_allowed"], "host": host},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of whole oracle steps for cpu_baseline (at least one step)")
    ap.add_argument("--no-threaded-oracle", action="store_true", help="skip the threaded oracle run")
    ap.add_argument("--ref-budget", type=float, default=100.0,
                    help="seconds of whole oracle steps for --impl reference (at least one step)")
    ap.add_argument("--oracle-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-budget", type=float, default=20.0, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-max-steps", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 512-simulation measurement")
    ap.add_argument("--no-collisions", action="store_true", help="skip the collision measurement")
    ap.add_argument("--no-pcg", action="store_true", help="skip the Jacobi-PCG measurement")
    ap.add_argument("--no-convergence", action="store_true", help="skip the relative-error measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the spline-bar and large-bar measurements")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--no-tune-cache", action="store_true", help="ignore the autotuner's cache (library defaults)")
    ap.add_argument("--leaf-size", type=int, default=0,
                    help="max vertices of a nested-dissection leaf (0 = the library default)")
    ap.add_argument("--solve-threads", type=int, default=0, help="threads per sweep block (0 = default)")
    ap.add_argument("--solve-item-kb", type=int, default=0, help="largest sweep work item in KB (0 = default)")
    ap.add_argument("--solve-items", type=int, default=0, help="work items per tree level (0 = default)")
    ap.add_argument("--solve-prefetch", type=int, default=0,
                    help="L2 prefetch distance of the sweeps in launches (0 = default, -1 = none)")
    ap.add_argument("--no-graph", action="store_true",
                    help="issue the step's kernels one by one (same kernels; for profilers that "
                         "cannot see inside graphs with conditional nodes)")
    args = ap.parse_args()
    if args.oracle_child:
        oracle_child(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank)), flush=True)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    line = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
