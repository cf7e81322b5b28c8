"""Filtered ordered-statistics decoding (filtered-OSD), plain and slow (TEST
INFRASTRUCTURE ONLY: only tests, the smoke check and the benchmark's CPU legs use it).

Paper Sec. 5 ("Filtered ordered statistics decoding" and its input, ranking,
submatrix and solver subsections) with the pre-decoder of Sec. 7.1:

1. pre-decoder: the first Relay leg (80 DMem-BP iterations with gamma_0); a shot
   whose first leg converges keeps that correction and is not post-processed;
2. otherwise 25 iterations of plain min-sum BP (Sec. 2.3 "Belief propagation
   decoding": DMem-BP with every gamma_j = 0, started afresh from the priors, no
   early exit) give the LLRs Lambda;
3. R = the faults with Lambda_j < Lambda_confident, in increasing Lambda_j (ties:
   increasing j); more than |R|_max of them is a failure;
4. x solves H_R x = sigma with x supported on the pivot columns of H_R taken left
   to right (the leftmost linearly independent columns; free columns 0); no solution
   is a failure;
5. F_j = x_r for j = R_r, zero elsewhere.

Step 4 is written as textbook Gauss-Jordan elimination to reduced row-echelon form
over GF(2), column by column from the left, on all M rows of H_R with sigma as an
augmented column.  The streaming "lifted" elimination the paper's solver uses
(Algorithm "Lifted Gauss-Jordan over F_2") reaches the same x: the set of leading
positions of any echelon basis of a row space is the same, and the solution
supported on those columns is unique.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .relay import RelayParams, dmem_trace, relay_decode

OK_PREDECODER = 0      # first Relay leg converged; its correction is kept
OK_OSD = 1             # filtered-OSD found a solution
FAIL_TOO_MANY = -1     # more than max_candidates faults below the threshold
FAIL_NO_SOLUTION = -2  # H_R x = sigma has no solution


@dataclass
class OSDParams:
    bp_iters: int = 25
    llr_confident: float = 4.0
    max_candidates: int = 500


def gf2_solve_leftmost(A: np.ndarray, y: np.ndarray):
    """x with A x = y over GF(2), supported on the pivot columns of RREF(A).

    Returns (x uint8 [n], consistent bool, pivots list).  Gauss-Jordan: for each
    column from the left, take the first remaining row with a 1 as pivot row, clear
    the column in every other row (and in y); rows left over must have y = 0.
    """
    A = np.array(A, dtype=np.uint8) & 1
    y = np.array(y, dtype=np.uint8) & 1
    m, n = A.shape
    row = 0
    piv = []
    for c in range(n):
        if row == m:
            break
        cand = np.nonzero(A[row:, c])[0]
        if cand.size == 0:
            continue
        r = row + int(cand[0])
        if r != row:
            A[[row, r]] = A[[r, row]]
            y[[row, r]] = y[[r, row]]
        hit = np.nonzero(A[:, c])[0]
        hit = hit[hit != row]
        A[hit] ^= A[row]
        y[hit] ^= y[row]
        piv.append(c)
        row += 1
    consistent = not y[row:].any()
    x = np.zeros(n, dtype=np.uint8)
    if consistent:
        for k, c in enumerate(piv):
            x[c] = y[k]
    return x, consistent, piv


def filtered_ranking(llr: np.ndarray, llr_confident: float) -> np.ndarray:
    """Indices j with llr_j < llr_confident, in increasing llr_j, ties by j."""
    llr = np.asarray(llr, dtype=np.float64)
    keep = np.nonzero(llr < llr_confident)[0]
    order = np.lexsort((keep, llr[keep]))      # primary key llr, secondary j
    return keep[order]


def filtered_osd(H: np.ndarray, sigma: np.ndarray, llr: np.ndarray, prm: OSDParams):
    """One shot: (F uint8 [N], status, |R|).  F is zero on failure."""
    H = np.asarray(H, dtype=np.uint8)
    N = H.shape[1]
    R = filtered_ranking(llr, prm.llr_confident)
    F = np.zeros(N, dtype=np.uint8)
    if R.size > prm.max_candidates:
        return F, FAIL_TOO_MANY, int(R.size)
    x, ok, _ = gf2_solve_leftmost(H[:, R], sigma)
    if not ok:
        return F, FAIL_NO_SOLUTION, int(R.size)
    F[R] = x
    return F, OK_OSD, int(R.size)


def bp_llrs(row_ptr, col_idx, priors, sigma, T: int = 25, precision: str = "f32"):
    """Marginals after T iterations of min-sum BP (gamma = 0), no early exit."""
    N = np.asarray(priors).size
    if T == 0:                               # no iteration: the prior LLRs themselves
        p = np.asarray(priors, dtype=np.float64)
        w = np.log((1.0 - p) / p)
        if precision != "f64":
            w = w.astype(np.float32).astype(np.float64)
        return np.repeat(w[None, :], np.asarray(sigma).shape[0], axis=0)
    Lam, _, _ = dmem_trace(row_ptr, col_idx, priors, np.zeros(N), sigma, T,
                           precision=precision, want_messages=False)
    return Lam[:, T - 1, :]


def first_leg_then_osd(H, row_ptr, col_idx, priors, gamma0_row, sigma, prm: OSDParams,
                       precision: str = "f32"):
    """The whole post-processed decoder on a batch sigma (uint8 [B, M]).

    Returns (F uint8 [B, N], status int32 [B], n_candidates int32 [B]).
    """
    sigma = np.ascontiguousarray(sigma, dtype=np.uint8)
    B = sigma.shape[0]
    pre = relay_decode(row_ptr, col_idx, priors, np.asarray(gamma0_row)[None, :], sigma,
                       RelayParams(legs_after_first=0, stop_after_solutions=1),
                       precision=precision)
    F = pre.corrections.copy()
    status = np.full(B, OK_PREDECODER, dtype=np.int32)
    ncand = np.zeros(B, dtype=np.int32)
    todo = np.nonzero(pre.converged == 0)[0]
    if todo.size:
        llr = bp_llrs(row_ptr, col_idx, priors, sigma[todo], prm.bp_iters, precision)
        for k, b in enumerate(todo):
            f, st, n = filtered_osd(H, sigma[b], llr[k], prm)
            status[b] = st
            ncand[b] = n
            if st == OK_OSD:
                F[b] = f
    return F, status, ncand
