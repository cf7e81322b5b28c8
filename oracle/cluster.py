"""Generalized union-find cluster decoder with a BP pre-decoder, plain and slow (TEST
INFRASTRUCTURE ONLY: only tests, the smoke check and the benchmark's CPU legs use it).

Paper Sec. 2.5 ("Cluster decoding", with "BP-UF decoding") and its FPGA form in Sec. 6
(input, initialisation, growth, merging, interior faults, validity, output), with the
pre-decoder of Sec. 7.1:

* input: after the first Relay leg fails, 25 iterations of plain min-sum BP give Lambda;
  faults with Lambda_j <= accept are applied as a partial correction F_pre, faults with
  accept < Lambda_j <= erase form the erasure set; sigma <- sigma_original + H F_pre;
* clusters are vertex sets of the Tanner graph (checks 0..M-1, then faults M..M+N-1),
  one per syndrome check and per erased fault;
* a cluster is valid when its syndrome lies in the image of H restricted to its checks
  (rows) and its interior faults (columns: faults whose every check is in the cluster);
* loop: take the first invalid cluster of the list, grow it by all neighbours of its
  vertices, merge into it every cluster it now intersects, test it; append it to the
  end of the list if still invalid;
* output: per cluster, the solution on its interior faults (columns in increasing
  fault index) with free columns 0; the correction is F_pre + the union of those.

The initial clusters come in the seed-extraction order of Sec. 6.3: the right-most set
bit of the initialisation bitmap first, where the bitmap lists check 0 left-most and the
fault nodes after the checks, i.e. in decreasing node index (the check and fault parts
are extracted independently; a cluster seeded by an erased fault has no interior fault
and no check, so it starts valid and never enters the invalid list).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .osd import bp_llrs, gf2_solve_leftmost
from .relay import RelayParams, relay_decode

OK_PREDECODER = 0    # first Relay leg converged; its correction is kept
OK_CLUSTER = 1       # every cluster valid; correction = F_pre + cluster solutions
FAIL_TOO_LARGE = -1  # a cluster exceeded max_cluster_faults interior faults
FAIL_TOO_MANY = -2   # more than max_clusters initial clusters


@dataclass
class ClusterParams:
    bp_iters: int = 25
    llr_accept: float = -4.0
    llr_erase: float = 2.0
    max_cluster_faults: int = 1024
    max_clusters: int = 128


def adjacency(H: np.ndarray):
    """Neighbour lists of the Tanner graph with checks 0..M-1 and faults M..M+N-1."""
    M, N = H.shape
    nb = []
    for i in range(M):
        nb.append(set((M + np.nonzero(H[i])[0]).tolist()))
    for j in range(N):
        nb.append(set(np.nonzero(H[:, j])[0].tolist()))
    return nb


def interior_faults(H: np.ndarray, V: set) -> list:
    """Faults of V whose every check lies in V, increasing index."""
    M = H.shape[0]
    out = []
    for v in sorted(V):
        if v >= M:
            j = v - M
            if all(i in V for i in np.nonzero(H[:, j])[0]):
                out.append(j)
    return out


def cluster_system(H: np.ndarray, sigma: np.ndarray, V: set):
    """(H restricted to the cluster's checks x interior faults, its syndrome, faults)."""
    M = H.shape[0]
    rows = sorted(v for v in V if v < M)
    cols = interior_faults(H, V)
    A = H[np.ix_(rows, cols)] if rows and cols else np.zeros((len(rows), len(cols)), np.uint8)
    return A, sigma[rows], cols


def is_valid(H, sigma, V) -> bool:
    A, y, _ = cluster_system(H, sigma, V)
    if A.shape[1] == 0:
        return not y.any()
    return gf2_solve_leftmost(A, y)[1]


def cluster_decode(H: np.ndarray, sigma: np.ndarray, erasures: np.ndarray,
                   max_cluster_faults: int = 1 << 30, max_clusters: int = 1 << 30, nb=None):
    """Union-find cluster decoding of (sigma, erasure set).  Returns (F, status, steps)."""
    H = np.asarray(H, dtype=np.uint8)
    M, N = H.shape
    nb = nb if nb is not None else adjacency(H)
    if int(np.count_nonzero(sigma)) + int(np.count_nonzero(erasures)) > max_clusters:
        return np.zeros(N, np.uint8), FAIL_TOO_MANY, 0
    seeds = np.concatenate([np.nonzero(sigma)[0][::-1], M + np.nonzero(erasures)[0][::-1]])
    clusters = {}                       # id -> vertex set
    order = []                          # invalid-cluster list (ids), first = next to grow
    for cid, v in enumerate(seeds.tolist()):
        clusters[cid] = {v}
    for cid in range(len(seeds)):       # initial validity test, in seed order
        if not is_valid(H, sigma, clusters[cid]):
            order.append(cid)
    steps = 0
    while order:
        cid = order.pop(0)
        V = clusters[cid]
        grown = set(V)
        for v in V:
            grown |= nb[v]
        for other in sorted(clusters):  # every other cluster in turn
            if other != cid and clusters[other] & grown:
                grown |= clusters.pop(other)
                if other in order:
                    order.remove(other)
        clusters[cid] = grown
        steps += 1
        if len(interior_faults(H, grown)) > max_cluster_faults:
            return np.zeros(N, np.uint8), FAIL_TOO_LARGE, steps
        if not is_valid(H, sigma, grown):
            order.append(cid)
    F = np.zeros(N, dtype=np.uint8)
    for cid in sorted(clusters):
        A, y, cols = cluster_system(H, sigma, clusters[cid])
        if cols:
            x, ok, _ = gf2_solve_leftmost(A, y)
            assert ok
            F[cols] |= x
    return F, OK_CLUSTER, steps


def bp_uf(H, sigma_original, llr, prm: ClusterParams):
    """BP-UF on one shot from pre-decoder marginals llr: (F, status, steps)."""
    H = np.asarray(H, dtype=np.uint8)
    llr = np.asarray(llr, dtype=np.float64)
    pre = (llr <= prm.llr_accept).astype(np.uint8)
    era = ((llr > prm.llr_accept) & (llr <= prm.llr_erase)).astype(np.uint8)
    sigma = (sigma_original.astype(np.int64) + H.astype(np.int64) @ pre) % 2
    F, st, steps = cluster_decode(H, sigma.astype(np.uint8), era, prm.max_cluster_faults,
                                  prm.max_clusters)
    return (F ^ pre) if st == OK_CLUSTER else np.zeros_like(F), st, steps


def first_leg_then_cluster(H, row_ptr, col_idx, priors, gamma0_row, sigma, prm: ClusterParams,
                           precision: str = "f32"):
    """First Relay leg on every shot; BP-UF on the shots it leaves unconverged.
    Returns (F uint8 [B, N], status int32 [B], steps int32 [B])."""
    sigma = np.ascontiguousarray(sigma, dtype=np.uint8)
    B = sigma.shape[0]
    pre = relay_decode(row_ptr, col_idx, priors, np.asarray(gamma0_row)[None, :], sigma,
                       RelayParams(legs_after_first=0, stop_after_solutions=1),
                       precision=precision)
    F = pre.corrections.copy()
    status = np.full(B, OK_PREDECODER, dtype=np.int32)
    steps = np.zeros(B, dtype=np.int32)
    todo = np.nonzero(pre.converged == 0)[0]
    if todo.size:
        llr = bp_llrs(row_ptr, col_idx, priors, sigma[todo], prm.bp_iters, precision)
        for k, b in enumerate(todo):
            f, st, n = bp_uf(H, sigma[b], llr[k], prm)
            status[b] = st
            steps[b] = n
            if st == OK_CLUSTER:
                F[b] = f
    return F, status, steps
