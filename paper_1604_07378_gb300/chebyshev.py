"""The spectral radius rho that Alg. 3's Chebyshev weights need, estimated
from a projective-dynamics run (Alg. 1 with the m = 0 direction).

Near its minimiser the projective-dynamics iteration x_{k+1} = x_k - A0^{-1}
grad g(x_k) is linear: x_k - x* shrinks by the spectral radius rho of
I - A0^{-1} H (H the Hessian of g at x*) per iteration, so the objective's
excess g_k - g* ~ rho^(2k), and so do its decrements d_k = g_k - g_{k+1}.
The estimate is the square root of the median ratio d_{k+1} / d_k over the
run's last iterations (the median guards against a line-search step that
does not take the full alpha = 1).  It needs only the per-iteration
objective values that sim_step reports.
"""
from __future__ import annotations

import numpy as np


def estimate_rho(g_values, tail: int = 12) -> float:
    """rho from the objective values g_0, g_1, ... of one projective-dynamics
    step (the iterations' g in order); uses the last `tail` decrements that
    are positive and above rounding."""
    g = np.asarray(g_values, dtype=np.float64)
    d = g[:-1] - g[1:]
    floor = 1e-13 * max(1.0, float(np.abs(g).max()))
    ok = np.flatnonzero(d > floor)
    if ok.size < 3:
        raise ValueError("too few decreasing iterations to estimate rho")
    d = d[ok[-(tail + 1):]]
    r = d[1:] / d[:-1]
    r = r[(r > 0.0) & (r < 1.0)]
    if r.size == 0:
        raise ValueError("the projective-dynamics run does not contract")
    return float(np.sqrt(np.median(r)))
