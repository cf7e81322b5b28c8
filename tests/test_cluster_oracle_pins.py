"""Pins of the cluster-decoder oracle (oracle/cluster.py), paper Sec. 2.5 and Sec. 6.

* a hand-traced run on a chain (two syndrome clusters grow in list order, fail, and
  merge on the fourth growth step into one valid cluster), fixing growth, merging, the
  first-in-first-out invalid list and the step count;
* validity against brute force on small random clusters;
* on detector models: every correction satisfies its syndrome, clusters end disjoint
  and valid, erased faults alone give valid empty clusters, and the caps fail.
"""
import numpy as np
import pytest

from oracle.cluster import (FAIL_TOO_LARGE, FAIL_TOO_MANY, OK_CLUSTER, OK_PREDECODER,
                            ClusterParams, adjacency, bp_uf, cluster_decode,
                            first_leg_then_cluster, interior_faults, is_valid)
from oracle.osd import bp_llrs
from workloads import BB72, gamma_table, phenomenological_dem, sample_faults, syndromes_of

from _brute import all_bitstrings


def test_hand_traced_chain():
    # c0 - f0 - c1 - f1 - c2, syndrome of f0 + f1
    H = np.array([[1, 0], [1, 1], [0, 1]], np.uint8)
    sigma = np.array([1, 0, 1], np.uint8)
    F, st, steps = cluster_decode(H, sigma, np.zeros(2, np.uint8))
    # c2's cluster grows to {c2,f1} (invalid), c0's to {c0,f0} (invalid), c2's to
    # {c2,f1,c1} (f1 interior, sigma (0,1) not in its image: invalid), c0's to
    # {c0,f0,c1}, which meets c2's cluster: merged, both faults interior, valid
    assert st == OK_CLUSTER and steps == 4
    assert F.tolist() == [1, 1]


def test_single_check_clusters_start_invalid_and_erasures_start_valid():
    H = np.array([[1, 0], [1, 1], [0, 1]], np.uint8)
    sig = np.array([0, 1, 0], np.uint8)
    assert not is_valid(H, sig, {1})
    assert is_valid(H, sig, {3})                        # an erased fault alone: empty system
    assert interior_faults(H, {0, 1, 3}) == [0]         # f0's checks c0, c1 both inside
    F, st, steps = cluster_decode(H, np.zeros(3, np.uint8), np.array([1, 1], np.uint8))
    assert st == OK_CLUSTER and steps == 0 and not F.any()


@pytest.mark.parametrize("seed", range(30))
def test_validity_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    M, N = int(rng.integers(3, 7)), int(rng.integers(3, 9))
    H = (rng.random((M, N)) < 0.4).astype(np.uint8)
    sigma = rng.integers(0, 2, M).astype(np.uint8)
    V = set(np.nonzero(rng.random(M + N) < 0.6)[0].tolist())
    rows = sorted(v for v in V if v < M)
    cols = [j for j in range(N) if M + j in V and all(i in V for i in np.nonzero(H[:, j])[0])]
    assert interior_faults(H, V) == cols
    X = all_bitstrings(len(cols)) if cols else np.zeros((1, 0), np.uint8)
    A = H[np.ix_(rows, cols)] if rows and cols else np.zeros((len(rows), len(cols)), np.uint8)
    ok = ((X.astype(int) @ A.T.astype(int)) % 2 == sigma[rows][None, :]).all(1).any()
    assert is_valid(H, sigma, V) == bool(ok)


def _problem(p, shots, seed):
    P = phenomenological_dem(BB72, 6, p)
    F = sample_faults(P.p, seed, shots)
    return P, F, syndromes_of(P.row_ptr, P.col_idx, F)


def test_cluster_corrections_satisfy_the_syndrome():
    P, F, s = _problem(0.02, 40, 3)
    nb = adjacency(P.H)
    for b in range(s.shape[0]):
        out, st, steps = cluster_decode(P.H, s[b], np.zeros(P.N, np.uint8), nb=nb)
        assert st == OK_CLUSTER
        assert (((P.H.astype(int) @ out) % 2) == s[b]).all()


def test_bp_uf_with_partial_correction_and_erasures():
    P, F, s = _problem(0.04, 30, 5)
    L = bp_llrs(P.row_ptr, P.col_idx, P.p, s)
    w = np.log(0.96 / 0.04)
    prm = ClusterParams(llr_accept=-0.5, llr_erase=w + 0.5, max_clusters=4000)
    n_era = 0
    for b in range(s.shape[0]):
        n_era += int(((L[b] > -0.5) & (L[b] <= w + 0.5)).sum())
        out, st, steps = bp_uf(P.H, s[b], L[b], prm)
        assert st == OK_CLUSTER
        assert (((P.H.astype(int) @ out) % 2) == s[b]).all()
    assert n_era > 0


def test_caps_fail():
    P, F, s = _problem(0.04, 10, 7)
    b = int(np.argmax(s.sum(1)))
    out, st, _ = cluster_decode(P.H, s[b], np.zeros(P.N, np.uint8), max_clusters=2)
    assert st == FAIL_TOO_MANY and not out.any()
    out, st, _ = cluster_decode(P.H, s[b], np.zeros(P.N, np.uint8), max_cluster_faults=1)
    assert st == FAIL_TOO_LARGE and not out.any()


def test_pipeline_keeps_first_leg_successes():
    P, F, s = _problem(0.05, 60, 9)
    g0 = gamma_table(P.N, 0, 0.125, -0.24, 0.66, 1)[0]
    Fo, st, steps = first_leg_then_cluster(P.H, P.row_ptr, P.col_idx, P.p, g0, s,
                                           ClusterParams(llr_accept=-0.5, llr_erase=3.5,
                                                         max_clusters=4000))
    assert (st == OK_PREDECODER).sum() > 0 and (st == OK_CLUSTER).sum() >= 5
    ok = st != FAIL_TOO_LARGE
    assert (((Fo[ok].astype(int) @ P.H.T.astype(int)) % 2) == s[ok]).all()
