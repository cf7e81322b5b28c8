"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/relay_oracle.c) against something other
than itself: exact min-sum marginals on trees by brute force, the closed-form
linear dynamics of DMem-BP when every check has degree two, the paper's
iteration bound for a syndrome that has no solution (App. A.3, Sec. 7.2),
brute-force minimum-weight decoding on tiny codes, and the syndrome invariant.
"""
import json
import os

import numpy as np
import pytest

from oracle.relay import RelayParams, dmem_trace, relay_decode
from workloads import (BB72, BB144, code_capacity_dem, gamma_table, gf2_nullspace,
                       phenomenological_dem, sample_faults, syndromes_of)

from _brute import (csr, min_weight, minsum_llr_exact, random_degree2_checks, random_tree)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _syndrome(H, F):
    return ((F.astype(np.int64) @ H.T.astype(np.int64)) % 2).astype(np.uint8)


# --------------------------------------------------------------------------------------
# Check and fault rules: exact on trees (gamma = 0 is MinSum BP, Sec. 2.3)
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_minsum_marginals_exact_on_trees(seed):
    rng = np.random.default_rng(seed)
    H = random_tree(rng, n_checks=int(rng.integers(3, 6)), max_new=2)
    M, N = H.shape
    assert N <= 16
    p = rng.uniform(0.02, 0.3, N)
    w = np.log((1 - p) / p)
    row_ptr, col_idx = csr(H)
    sig = rng.integers(0, 2, (4, M)).astype(np.uint8)
    T = 2 * (M + N)
    for prec, tol in (("f64", 1e-12), ("f32", 2e-5)):
        Lam, _, _ = dmem_trace(row_ptr, col_idx, p, np.zeros(N), sig, T, precision=prec)
        for b in range(sig.shape[0]):
            exact = minsum_llr_exact(H, w, sig[b])
            assert np.isfinite(exact).all()
            np.testing.assert_allclose(Lam[b, -1], exact, rtol=tol, atol=tol)
            # converged: the last two iterations agree
            np.testing.assert_allclose(Lam[b, -1], Lam[b, -2], rtol=tol, atol=tol)


# --------------------------------------------------------------------------------------
# Memory rule, excluded sums, syndrome sign: closed form when checks have degree two
# --------------------------------------------------------------------------------------
def _degree2_linear_model(H, w, gamma_rows, sigma, legs_T, warm_mode):
    """DMem-BP/Relay on a graph whose checks have degree two, as an affine map.

    With two faults per check the min over the excluded set has one element, so
    mu_e(t) = (-1)^{sigma_i} nu_{partner(e)}(t-1).  In matrix form over edges:
      mu(t)     = S P nu(t-1)
      lambda(t) = (1-gamma) lambda0 + gamma Lambda(t-1)
      Lambda(t) = lambda(t) + V mu(t)
      nu(t)     = V^T lambda(t) + (V^T V - I) mu(t)
    with P the partner permutation, S the syndrome signs and V the fault/edge
    incidence.  Legs are chained as in Sec. 2.3 ("Relay chaining").
    """
    M, N = H.shape
    rows, cols = np.nonzero(H)
    E = rows.size
    P = np.zeros((E, E))
    for i in range(M):
        a, b = np.nonzero(rows == i)[0]
        P[a, b] = P[b, a] = 1
    S = np.diag(np.where(sigma[rows] == 1, -1.0, 1.0))
    V = np.zeros((N, E))
    V[cols, np.arange(E)] = 1
    lam0 = w.copy()
    Lam = lam0.copy()
    history = []
    for leg, T in enumerate(legs_T):
        g = gamma_rows[leg]
        if leg > 0:
            lam0 = Lam.copy() if warm_mode == 0 else w.copy()
        nu = V.T @ lam0
        for _ in range(T):
            mu = S @ P @ nu
            lam = (1 - g) * lam0 + g * Lam
            Lam = lam + V @ mu
            nu = V.T @ lam + (V.T @ V - np.eye(E)) @ mu
            history.append((Lam.copy(), nu.copy(), mu.copy()))
    return history


@pytest.mark.parametrize("seed", range(4))
def test_memory_rule_closed_form_degree2(seed):
    rng = np.random.default_rng(100 + seed)
    N, M = 12, 16
    H = random_degree2_checks(rng, N, M)
    row_ptr, col_idx = csr(H)
    p = rng.uniform(0.05, 0.45, N)
    w = np.log((1 - p) / p)
    gam = np.float32(rng.uniform(-0.24, 0.66, N)).astype(np.float64)
    sig = rng.integers(0, 2, M).astype(np.uint8)
    T = 10
    hist = _degree2_linear_model(H, w, [gam], sig, [T], 0)
    Lam, nu, mu = dmem_trace(row_ptr, col_idx, p, gam, sig[None, :], T)
    for t in range(T):
        L_ref, nu_ref, mu_ref = hist[t]
        np.testing.assert_allclose(Lam[0, t], L_ref, rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(nu[0, t], nu_ref, rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(mu[0, t], mu_ref, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("warm_mode", [0, 1])
def test_relay_chaining_closed_form_degree2(warm_mode):
    """Chained legs on an unsatisfiable syndrome follow the warm-start formulas."""
    rng = np.random.default_rng(7)
    N, M = 10, 14
    H = random_degree2_checks(rng, N, M)
    row_ptr, col_idx = csr(H)
    left = gf2_nullspace(H.T)
    assert left.shape[0] > 0
    y = left[0]
    sig = np.zeros(M, dtype=np.uint8)
    sig[np.nonzero(y)[0][0]] = 1                   # y . sigma = 1: no F has H F = sigma
    p = rng.uniform(0.05, 0.3, N)
    w = np.log((1 - p) / p)
    R, T1, T2 = 3, 5, 4
    gam = gamma_table(N, R, 0.125, -0.24, 0.66, seed=3)
    prm = RelayParams(legs_after_first=R, iters_first=T1, iters_later=T2,
                      stop_after_solutions=1, warm_start_mode=warm_mode)
    res = relay_decode(row_ptr, col_idx, p, gam, sig[None, :], prm, want_marginals=True)
    assert res.converged[0] == 0 and res.legs[0] == R + 1 and res.iters[0] == T1 + R * T2
    hist = _degree2_linear_model(H, w, gam, sig, [T1] + [T2] * R, warm_mode)
    np.testing.assert_allclose(res.final_marginals[0], hist[-1][0], rtol=1e-10, atol=1e-10)
    assert (res.corrections[0] == (hist[-1][0] < 0)).all()


# --------------------------------------------------------------------------------------
# Leg bookkeeping: the paper's maximum runtime (App. A.3 parameters, Sec. 7.2 bound)
# --------------------------------------------------------------------------------------
def _unsatisfiable_syndrome(H):
    y = gf2_nullspace(H.T)[0]
    s = np.zeros(H.shape[0], dtype=np.uint8)
    s[np.nonzero(y)[0][0]] = 1
    return s


def test_unsolvable_syndrome_runs_every_leg_to_paper_bound():
    g = json.load(open(os.path.join(GOLDEN, "relay_parameters_appA3.json")))
    P = code_capacity_dem(BB72, 0.05)
    sig = _unsatisfiable_syndrome(P.H)[None, :]
    gam = gamma_table(P.N, g["R"], g["gamma0"], *g["gamma_range_gross"], seed=0)
    prm = RelayParams(legs_after_first=g["R"], iters_first=g["T_first_leg"],
                      iters_later=g["T_later_legs"], stop_after_solutions=g["S"])
    res = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, prm)
    # the maximum runtime of Sec. 7.2 is alpha = 2 FPGA cycles per iteration
    assert res.iters[0] * g["fpga_cycles_per_iteration_alpha"] == g["two_gross_max_runtime_cycles"]
    assert res.legs[0] == g["R"] + 1 and res.converged[0] == 0
    # an iteration budget stops it early, part-way through leg 17
    prm.max_total_iters = 1000
    res = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, prm)
    assert res.iters[0] == 1000 and res.legs[0] == 17 and res.converged[0] == 0


@pytest.mark.parametrize("S", [1, 5])
def test_zero_syndrome(S):
    P = phenomenological_dem(BB72, 2, 0.01)
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, seed=0)
    res = relay_decode(P.row_ptr, P.col_idx, P.p, gam, np.zeros((3, P.M), np.uint8),
                       RelayParams(stop_after_solutions=S))
    assert (res.iters == S).all() and (res.legs == S).all() and (res.converged == 1).all()
    assert res.corrections.sum() == 0


# --------------------------------------------------------------------------------------
# Solutions: syndrome invariant and minimum weight by brute force
# --------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32", "f16s"])
def test_every_converged_correction_satisfies_syndrome(prec):
    P = code_capacity_dem(BB72, 0.05)
    F = sample_faults(P.p, 0, 600)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, seed=0)
    res = relay_decode(P.row_ptr, P.col_idx, P.p, gam, s, RelayParams(stop_after_solutions=5),
                       precision=prec)
    ok = res.converged == 1
    assert ok.mean() > 0.95
    assert (_syndrome(P.H, res.corrections[ok]) == s[ok]).all()


def test_single_faults_are_decoded_exactly():
    """A single fault has a unique minimum-weight explanation in the [[72,12,6]] code."""
    P = code_capacity_dem(BB72, 0.05)
    F = np.eye(P.N, dtype=np.uint8)
    s = _syndrome(P.H, F)
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, seed=0)
    for prec in ("f64", "f32", "f16s"):
        res = relay_decode(P.row_ptr, P.col_idx, P.p, gam, s, RelayParams(stop_after_solutions=5),
                           precision=prec)
        assert (res.converged == 1).all()
        assert (res.corrections == F).all()


@pytest.mark.parametrize("seed", range(3))
def test_relay_weight_is_never_below_brute_force_minimum(seed):
    rng = np.random.default_rng(40 + seed)
    M, N = 8, 15
    H = np.zeros((M, N), dtype=np.uint8)
    for j in range(N):
        H[rng.choice(M, int(rng.integers(2, 4)), replace=False), j] = 1
    row_ptr, col_idx = csr(H)
    p = np.full(N, 0.08)
    w = np.log((1 - p) / p)
    F = (rng.random((40, N)) < 0.12).astype(np.uint8)
    s = _syndrome(H, F)
    gam = gamma_table(N, 300, 0.125, -0.24, 0.66, seed=seed)
    res = relay_decode(row_ptr, col_idx, p, gam, s, RelayParams(stop_after_solutions=5))
    equal = 0
    assert res.converged.mean() >= 0.8
    for b in np.nonzero(res.converged)[0]:
        wmin = min_weight(H, w, s[b])
        assert (_syndrome(H, res.corrections[b:b + 1])[0] == s[b]).all()
        wr = float(res.corrections[b] @ w)
        assert wr >= wmin - 1e-9
        equal += abs(wr - wmin) < 1e-9
    # Relay is a heuristic: equality is common but not guaranteed
    assert equal >= 0.5 * res.converged.sum()


def test_more_solutions_never_increase_the_weight():
    P = phenomenological_dem(BB72, 3, 0.02)
    F = sample_faults(P.p, 4, 300)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, seed=1)
    w = np.log((1 - P.p) / P.p)
    r1 = relay_decode(P.row_ptr, P.col_idx, P.p, gam, s, RelayParams(stop_after_solutions=1))
    r5 = relay_decode(P.row_ptr, P.col_idx, P.p, gam, s, RelayParams(stop_after_solutions=5))
    both = (r1.converged == 1) & (r5.converged == 1)
    assert (r5.corrections[both] @ w <= r1.corrections[both] @ w + 1e-9).all()


# --------------------------------------------------------------------------------------
# Precision mirrors stay close to the FP64 oracle over the first iterations
# --------------------------------------------------------------------------------------
def test_precision_mirrors_track_fp64():
    P = phenomenological_dem(BB144, 12, 0.003)
    F = sample_faults(P.p, 1, 16)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    gam0 = np.full(P.N, 0.125)
    ref, nu_ref, _ = dmem_trace(P.row_ptr, P.col_idx, P.p, gam0, s, 10)
    for prec, tol in (("f32", 1e-5), ("f16s", 4e-3)):
        L, nu, _ = dmem_trace(P.row_ptr, P.col_idx, P.p, gam0, s, 10, precision=prec)
        err = np.abs(L - ref) / np.maximum(1.0, np.abs(ref))
        assert err.max() < tol, (prec, err.max())
        if prec == "f16s":
            assert (nu.astype(np.float16).astype(np.float64) == nu).all()


# --------------------------------------------------------------------------------------
# The benchmark's timed build (-O3) computes exactly what the parity build computes
# --------------------------------------------------------------------------------------
def test_timed_O3_build_equals_the_parity_build():
    """oracle/build.py's f64_O3 library (the CPU baseline the benchmark times) keeps
    -ffp-contract=off and no fast-math, so every output equals the -O2 build's, on
    gross-code shots at p = 0.02 that run many legs, with final marginals compared bit
    for bit and a single thread against all threads."""
    P = phenomenological_dem(BB144, 12, 0.02)
    F = sample_faults(P.p, 4, 48)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, 4)
    prm = RelayParams(stop_after_solutions=5, max_total_iters=600)
    a = relay_decode(P.row_ptr, P.col_idx, P.p, gam, s, prm, precision="f64",
                     want_marginals=True)
    b = relay_decode(P.row_ptr, P.col_idx, P.p, gam, s, prm, precision="f64_O3",
                     want_marginals=True, nthreads=1)
    assert a.legs.max() > 2
    for x, y in ((a.corrections, b.corrections), (a.legs, b.legs), (a.converged, b.converged),
                 (a.iters, b.iters)):
        assert np.array_equal(x, y)
    assert np.array_equal(a.final_marginals.view(np.uint64), b.final_marginals.view(np.uint64))
