"""Pins of the filtered-OSD oracle (oracle/osd.py), paper Sec. 5.

* the GF(2) solve against brute-force enumeration: consistency, the solution, its
  support on the leftmost independent columns (found by rank increments), and that it
  is the only solution with that support;
* the paper's streaming elimination (Algorithm "Lifted Gauss-Jordan over F_2": rows
  streamed, pivots locked at their leftmost 1, then back substitution) written out
  here independently gives the same solution on larger random systems, with the rows
  in any order;
* the same elimination with several rows in flight (the kernels' scheme: each round
  reduces every row in flight by the stored rows, then stores, for each free leading
  column met, the row of the lowest slot, the others going back for more reduction)
  reaches the same solution and the same verdict with 1, 4 or 32 slots;
* the ranking: strict threshold, increasing LLR, ties by fault index (the broadcast
  insertion sorter keeps equal keys in arrival order, and the LLRs arrive by index);
* the pipeline on a detector model: every OSD correction satisfies its syndrome and is
  supported on R, first-leg successes are left as they are, and the candidate cap fails.
"""
import numpy as np
import pytest

from oracle.osd import (FAIL_NO_SOLUTION, FAIL_TOO_MANY, OK_OSD, OK_PREDECODER, OSDParams,
                        bp_llrs, filtered_osd, filtered_ranking, first_leg_then_osd,
                        gf2_solve_leftmost)
from workloads import (BB72, gamma_table, phenomenological_dem, sample_faults, syndromes_of)

from _brute import all_bitstrings


def _rank(A):
    A = (np.array(A, dtype=np.uint8) & 1).copy()
    r = 0
    m, n = A.shape
    for c in range(n):
        rows = np.nonzero(A[r:, c])[0]
        if rows.size == 0:
            continue
        p = r + rows[0]
        A[[r, p]] = A[[p, r]]
        hit = np.nonzero(A[:, c])[0]
        A[hit[hit != r]] ^= A[r]
        r += 1
        if r == m:
            break
    return r


def _leftmost_independent(A):
    cols, rk = [], 0
    for c in range(A.shape[1]):
        k = _rank(A[:, :c + 1])
        if k > rk:
            cols.append(c)
            rk = k
    return cols


@pytest.mark.parametrize("seed", range(40))
def test_gf2_solve_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(1, 8)), int(rng.integers(1, 11))
    A = (rng.random((m, n)) < rng.uniform(0.2, 0.6)).astype(np.uint8)
    y = rng.integers(0, 2, m).astype(np.uint8)
    if seed % 3 == 0:                                  # a consistent right-hand side
        y = (A.astype(int) @ rng.integers(0, 2, n)) % 2
    x, ok, piv = gf2_solve_leftmost(A, y)
    X = all_bitstrings(n)
    sols = X[((X.astype(int) @ A.T.astype(int)) % 2 == y[None, :]).all(1)]
    assert ok == (sols.shape[0] > 0)
    assert piv == _leftmost_independent(A)
    if ok:
        assert ((A.astype(int) @ x) % 2 == y).all()
        off = np.ones(n, bool)
        off[piv] = False
        on_piv = sols[~sols[:, off].any(1)] if off.any() else sols
        assert on_piv.shape[0] == 1 and (on_piv[0] == x).all()


def _lifted_gauss_jordan(A, y):
    """Rows streamed in order; a row is reduced by the locked pivot rows until its
    leftmost 1 is an unlocked column, where it is stored; then back substitution."""
    m, n = A.shape
    up = np.zeros((n, n), dtype=np.uint8)
    spec = np.zeros(n, dtype=np.uint8)
    locked = np.zeros(n, dtype=bool)
    for i in range(m):
        r, s = A[i].copy(), int(y[i])
        while r.any():
            p = int(np.argmax(r))
            if not locked[p]:
                up[p], spec[p], locked[p] = r, s, True
                break
            r ^= up[p]
            s ^= int(spec[p])
        else:
            if s:
                return None
    x = np.zeros(n, dtype=np.uint8)
    for p in range(n - 1, -1, -1):
        if locked[p]:
            x[p] = (spec[p] + int((up[p, p + 1:] & x[p + 1:]).sum())) % 2
    return x


@pytest.mark.parametrize("seed", range(12))
def test_streaming_elimination_reaches_the_same_solution(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(20, 80)), int(rng.integers(10, 60))
    A = (rng.random((m, n)) < 0.08).astype(np.uint8)
    y = (A.astype(int) @ (rng.random(n) < 0.2)) % 2
    if seed % 4 == 3:
        y[int(rng.integers(0, m))] ^= 1                # usually inconsistent
    x, ok, _ = gf2_solve_leftmost(A, y)
    for order in (np.arange(m), rng.permutation(m)):
        z = _lifted_gauss_jordan(A[order], y[order])
        assert (z is not None) == ok
        if ok:
            assert (z == x).all()


def _rounds_of_rows(A, y, slots):
    """Rows taken from the stream by `slots` slots; per round every slot's row is reduced
    by the stored rows (which stay fixed during the round) until it is 0 or leads with a
    free column; a zero row with right-hand side 1 means no solution; for each free
    leading column, the row of the lowest slot leading with it is stored; slots whose row
    was stored or was 0 take the next rows.  Then back substitution."""
    m, n = A.shape
    up = np.zeros((n, n), dtype=np.uint8)
    spec = np.zeros(n, dtype=np.uint8)
    locked = np.zeros(n, dtype=bool)
    cur = [k if k < m else -1 for k in range(slots)]
    rows = [A[k].copy() if k < m else None for k in range(slots)]
    rhs = [int(y[k]) if k < m else 0 for k in range(slots)]
    nxt = slots
    while any(c >= 0 for c in cur):
        lead = [-1] * slots
        for k in range(slots):
            if cur[k] < 0:
                continue
            while rows[k].any():
                p = int(np.argmax(rows[k]))
                lead[k] = p
                if not locked[p]:
                    break
                rows[k] ^= up[p]
                rhs[k] ^= int(spec[p])
            else:
                lead[k] = -1
        done = []
        for k in range(slots):
            if cur[k] >= 0 and lead[k] < 0:
                if rhs[k]:
                    return None
                done.append(k)
        for k in range(slots):
            if cur[k] >= 0 and lead[k] >= 0 and lead[k] not in lead[:k]:
                up[lead[k]], spec[lead[k]], locked[lead[k]] = rows[k], rhs[k], True
                done.append(k)
        for k in sorted(done):
            cur[k] = nxt if nxt < m else -1
            if cur[k] >= 0:
                rows[k], rhs[k] = A[nxt].copy(), int(y[nxt])
            nxt += 1
    x = np.zeros(n, dtype=np.uint8)
    for p in range(n - 1, -1, -1):
        if locked[p]:
            x[p] = (spec[p] + int((up[p, p + 1:] & x[p + 1:]).sum())) % 2
    return x


@pytest.mark.parametrize("seed", range(12))
def test_rows_in_flight_reach_the_same_solution(seed):
    rng = np.random.default_rng(300 + seed)
    m, n = int(rng.integers(20, 120)), int(rng.integers(10, 90))
    A = (rng.random((m, n)) < 0.06).astype(np.uint8)
    y = (A.astype(int) @ (rng.random(n) < 0.2)) % 2
    if seed % 4 == 3:
        y[int(rng.integers(0, m))] ^= 1                # usually inconsistent
    x, ok, _ = gf2_solve_leftmost(A, y)
    for slots in (1, 4, 32):
        z = _rounds_of_rows(A, y, slots)
        assert (z is not None) == ok
        if ok:
            assert (z == x).all()


def test_ranking_threshold_order_and_ties():
    llr = np.array([3.0, -1.0, 2.0, -1.0, 5.0, 2.0, 4.0, -7.5])
    R = filtered_ranking(llr, 4.0)
    assert R.tolist() == [7, 1, 3, 2, 5, 0]            # strict <, increasing, ties by j
    assert filtered_ranking(llr, -7.5).size == 0


def test_square_invertible_system_gives_the_inverse_solution():
    rng = np.random.default_rng(7)
    while True:
        A = rng.integers(0, 2, (9, 9)).astype(np.uint8)
        if _rank(A) == 9:
            break
    x0 = rng.integers(0, 2, 9).astype(np.uint8)
    x, ok, piv = gf2_solve_leftmost(A, (A.astype(int) @ x0) % 2)
    assert ok and piv == list(range(9)) and (x == x0).all()


def _detector_problem(p, shots, seed):
    P = phenomenological_dem(BB72, 6, p)
    F = sample_faults(P.p, seed, shots)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    return P, F, s


def test_filtered_osd_solutions_satisfy_the_syndrome_on_R():
    P, F, s = _detector_problem(0.04, 60, 3)
    L = bp_llrs(P.row_ptr, P.col_idx, P.p, s)
    n_ok = 0
    for b in range(s.shape[0]):
        f, st, n = filtered_osd(P.H, s[b], L[b], OSDParams(llr_confident=4.0))
        R = filtered_ranking(L[b], 4.0)
        assert n == R.size
        if st == OK_OSD:
            n_ok += 1
            assert ((P.H.astype(int) @ f) % 2 == s[b]).all()
            assert not np.delete(f, R).any()
        else:
            assert st == FAIL_NO_SOLUTION and not f.any()
    assert n_ok >= 40


def test_candidate_cap_fails_and_zero_syndrome_solves():
    P, F, s = _detector_problem(0.04, 4, 5)
    L = bp_llrs(P.row_ptr, P.col_idx, P.p, s)
    f, st, n = filtered_osd(P.H, s[0], L[0], OSDParams(llr_confident=1e9, max_candidates=10))
    assert st == FAIL_TOO_MANY and n == P.N and not f.any()
    f, st, n = filtered_osd(P.H, np.zeros(P.M, np.uint8), L[0],
                            OSDParams(llr_confident=1e9, max_candidates=P.N))
    assert st == OK_OSD and not f.any()
    f, st, n = filtered_osd(P.H, s[0] | 1, L[0], OSDParams(llr_confident=-1e9))
    assert st == FAIL_NO_SOLUTION and n == 0


def test_pipeline_keeps_first_leg_successes():
    P, F, s = _detector_problem(0.05, 80, 9)
    g0 = gamma_table(P.N, 0, 0.125, -0.24, 0.66, 1)[0]
    Fo, st, nc = first_leg_then_osd(P.H, P.row_ptr, P.col_idx, P.p, g0, s,
                                    OSDParams(llr_confident=4.0))
    from oracle.relay import RelayParams, relay_decode
    pre = relay_decode(P.row_ptr, P.col_idx, P.p, g0[None, :], s,
                       RelayParams(legs_after_first=0), precision="f32")
    conv = pre.converged == 1
    assert (st[conv] == OK_PREDECODER).all() and (Fo[conv] == pre.corrections[conv]).all()
    assert (~conv).sum() >= 5 and (st[~conv] != OK_PREDECODER).all()
    ok = st == OK_OSD
    assert ok.any()
    assert (((Fo[ok].astype(int) @ P.H.T.astype(int)) % 2) == s[ok]).all()
