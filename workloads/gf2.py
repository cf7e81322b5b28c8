"""Small dense linear algebra over F2 (numpy uint8), used only to build and check inputs.

Matrices here are at most a few hundred rows (code check matrices), so plain
row reduction is fast enough.
"""
from __future__ import annotations

import numpy as np


def gf2_rref(a: np.ndarray):
    """Reduced row-echelon form over F2.

    Returns ``(R, pivots)`` where ``R`` is the reduced matrix (same shape) and
    ``pivots`` lists the pivot column of each non-zero row, in row order.
    """
    r = (np.asarray(a, dtype=np.uint8) & 1).copy()
    rows, cols = r.shape
    pivots = []
    row = 0
    for c in range(cols):
        if row >= rows:
            break
        hits = np.nonzero(r[row:, c])[0]
        if hits.size == 0:
            continue
        p = row + hits[0]
        if p != row:
            r[[row, p]] = r[[p, row]]
        others = np.nonzero(r[:, c])[0]
        others = others[others != row]
        if others.size:
            r[others] ^= r[row]
        pivots.append(c)
        row += 1
    return r, pivots


def gf2_rank(a: np.ndarray) -> int:
    """Rank over F2."""
    return len(gf2_rref(a)[1])


def gf2_nullspace(a: np.ndarray) -> np.ndarray:
    """Basis of {x : a x = 0} over F2, one basis vector per row."""
    a = np.asarray(a, dtype=np.uint8) & 1
    n = a.shape[1]
    r, pivots = gf2_rref(a)
    free = [c for c in range(n) if c not in set(pivots)]
    basis = np.zeros((len(free), n), dtype=np.uint8)
    for k, f in enumerate(free):
        basis[k, f] = 1
        for row, pc in enumerate(pivots):
            if r[row, f]:
                basis[k, pc] = 1
    return basis
