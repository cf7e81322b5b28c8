"""Brute-force references and small graph generators for pinning the oracle.

These enumerate all 2^N fault sets, so they are only for N <= 16.
"""
from __future__ import annotations

import numpy as np


def all_bitstrings(n: int) -> np.ndarray:
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


def feasible(H: np.ndarray, sigma: np.ndarray):
    """All F with H F = sigma (mod 2), as uint8 [K, N]."""
    F = all_bitstrings(H.shape[1])
    s = (F.astype(np.int64) @ H.T.astype(np.int64)) % 2
    return F[(s == sigma[None, :]).all(1)]


def minsum_llr_exact(H, w, sigma):
    """min_{F: HF=sigma, F_j=1} w.F - min_{F: HF=sigma, F_j=0} w.F (inf if one side is empty)."""
    F = feasible(H, sigma)
    cost = F.astype(np.float64) @ np.asarray(w, dtype=np.float64)
    out = np.empty(H.shape[1])
    for j in range(H.shape[1]):
        c1 = cost[F[:, j] == 1]
        c0 = cost[F[:, j] == 0]
        a = c1.min() if c1.size else np.inf
        b = c0.min() if c0.size else np.inf
        out[j] = a - b
    return out


def sumproduct_llr_exact(H, p, sigma):
    """log P(F_j = 0 | sigma) - log P(F_j = 1 | sigma) under independent faults."""
    F = feasible(H, sigma)
    p = np.asarray(p, dtype=np.float64)
    logw = (F * np.log(p)[None, :] + (1 - F) * np.log1p(-p)[None, :]).sum(1)
    out = np.empty(H.shape[1])
    for j in range(H.shape[1]):
        a = np.logaddexp.reduce(logw[F[:, j] == 0]) if (F[:, j] == 0).any() else -np.inf
        b = np.logaddexp.reduce(logw[F[:, j] == 1]) if (F[:, j] == 1).any() else -np.inf
        out[j] = a - b
    return out


def min_weight(H, w, sigma):
    F = feasible(H, sigma)
    if F.shape[0] == 0:
        return np.inf
    return float((F.astype(np.float64) @ np.asarray(w, dtype=np.float64)).min())


def random_tree(rng, n_checks: int, max_new: int = 3) -> np.ndarray:
    """Random bipartite tree with every check of degree >= 2 (dense H, checks x faults).

    Grown from one fault: each new check attaches to one existing fault and to
    1..max_new new faults, so the Tanner graph stays acyclic.
    """
    edges = []
    n_vars = 1
    for c in range(n_checks):
        anchor = int(rng.integers(0, n_vars))
        k = int(rng.integers(1, max_new + 1))
        edges.append((c, anchor))
        for _ in range(k):
            edges.append((c, n_vars))
            n_vars += 1
    H = np.zeros((n_checks, n_vars), dtype=np.uint8)
    for c, v in edges:
        H[c, v] = 1
    return H


def random_degree2_checks(rng, n_vars: int, n_checks: int) -> np.ndarray:
    """Random graph whose checks all have exactly two faults (distinct pairs)."""
    pairs = set()
    while len(pairs) < n_checks:
        a, b = rng.choice(n_vars, 2, replace=False)
        pairs.add((min(a, b), max(a, b)))
    H = np.zeros((n_checks, n_vars), dtype=np.uint8)
    for c, (a, b) in enumerate(sorted(pairs)):
        H[c, a] = H[c, b] = 1
    return H


def csr(H):
    rows, cols = np.nonzero(H)
    row_ptr = np.zeros(H.shape[0] + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), cols.astype(np.int32)
