"""Latency-tail conditions for real-time decoding (paper Sec. 2.2, Eq. latency-tail-
requirement and Eq. latency-tail-slowdown; applied to Relay in Sec. 7.2).

A decoder finishes within T_ref with probability 1 - eps and always within T_max;
syndromes of one code block arrive every T_gen.  With C code blocks the backlog
stays bounded if T_ref < T_gen and eps * C * L < 1, where
L = ceil((T_max - T_ref) / (T_gen - T_ref)), and the mean slowdown then satisfies
<R> < 1 + T_ref / T_gen + 2 gamma / (1 - gamma), gamma = eps * C * L.
Times may be in any unit (FPGA cycles in the paper; here usually DMem-BP
iterations, taken from the decoder's per-shot iteration counts).
"""
from __future__ import annotations

import math

import numpy as np


def tail_probability(iters, t_ref: float) -> float:
    """eps: fraction of decoding runs that need more than t_ref."""
    it = np.asarray(iters)
    return float((it > t_ref).mean()) if it.size else 0.0


def layers(t_ref: float, t_gen: float, t_max: float) -> int:
    """L = ceil((T_max - T_ref) / (T_gen - T_ref)): idle layers a slow run inserts."""
    if not t_ref < t_gen:
        raise ValueError("needs T_ref < T_gen")
    return max(1, math.ceil((t_max - t_ref) / (t_gen - t_ref)))


def condition(eps: float, C: int, t_ref: float, t_gen: float, t_max: float):
    """(holds, L, gamma) for the latency-tail requirement eps * C * L < 1."""
    L = layers(t_ref, t_gen, t_max)
    gamma = eps * C * L
    return gamma < 1.0, L, gamma


def max_code_blocks(eps: float, t_ref: float, t_gen: float, t_max: float):
    """Largest C with eps * C * L < 1; None when eps = 0 (every C satisfies it)."""
    L = layers(t_ref, t_gen, t_max)
    if eps <= 0:
        return None
    c = math.ceil(1.0 / (eps * L)) - 1
    return max(c, 0)


def slowdown_bound(eps: float, C: int, t_ref: float, t_gen: float, t_max: float):
    """1 + T_ref/T_gen + 2 gamma / (1 - gamma); None when the requirement fails (the
    derivation gives no bound there)."""
    ok, L, gamma = condition(eps, C, t_ref, t_gen, t_max)
    if not ok:
        return None
    return 1.0 + t_ref / t_gen + 2.0 * gamma / (1.0 - gamma)


def report(iters, t_ref: float, t_gen: float, t_max: float, C: int, cycles_per_iter: float = 1.0):
    """Summary of a measured iteration distribution (times scaled by cycles_per_iter)."""
    it = np.asarray(iters, dtype=np.float64) * cycles_per_iter
    eps = tail_probability(it, t_ref)
    ok, L, gamma = condition(eps, C, t_ref, t_gen, t_max)
    return {"eps": eps, "L": L, "gamma": gamma, "holds": ok,
            "max_code_blocks": max_code_blocks(eps, t_ref, t_gen, t_max),
            "slowdown_bound": slowdown_bound(eps, C, t_ref, t_gen, t_max),
            "max_time": float(it.max()) if it.size else 0.0,
            "quantiles": {q: float(np.quantile(it, q)) for q in (0.5, 0.9, 0.99, 0.999)}
            if it.size else {}}
