"""Shared helpers of the GPU parity tests: build a handle and an oracle
problem from the same seeded workload."""
import numpy as np

from oracle import hqn_oracle as O
from paper_1604_07378_gb300 import workloads as W


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def sim_for(w, precision, **kw):
    from paper_1604_07378_gb300 import hqn
    return hqn.Sim.from_workload(w, precision=precision, **kw)


def problem_for(w):
    return O.problem_from_workload(w)


def perturbed(w, scale, seed):
    """A seeded state near the workload's current state (clamped vertices fixed)."""
    rng = np.random.default_rng(seed)
    x = w.q_cur + scale * rng.normal(size=w.q_cur.shape)
    x[w.clamped.astype(bool)] = w.q_cur[w.clamped.astype(bool)]
    return x


def small_workloads():
    """Small cases of each measured workload family (each spans several
    thread blocks and several supernode levels, with ragged tails)."""
    out = [W.bar_4x4x16_fp64()]
    out.append(W.lattice_workload((7, 6, 9), W.Material(W.STVK, 5e5, 0.4), clamp_axis=2, seed=11,
                                  v_range=0.5, name="lat7x6x9_stvk"))
    out.append(W.lattice_workload((7, 6, 9), W.Material(W.NEOHOOKEAN, 5e5, 0.4), clamp_axis=2,
                                  seed=12, v_range=0.5, name="lat7x6x9_nh"))
    out.append(W.spline_bar_80x40x40(scale=8))
    return out
