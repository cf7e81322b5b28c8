"""Pins of the soft DMem-BP oracle (oracle/soft_dmem_oracle.c).

* sum-product with gamma = 0 and alpha = 1 is exact on trees: the marginals equal
  the brute-force posterior log-likelihood ratios;
* with every check of degree two, 2 atanh(tanh(x/2)) = x makes the iteration an
  affine map whose matrix form fixes alpha_t, the memory rule and the signs;
* the hand-written reverse pass equals central finite differences of the loss.
"""
import numpy as np
import pytest

from oracle.soft import soft_dmem
from workloads import BB72, code_capacity_dem, sample_faults, syndromes_of

from _brute import csr, random_degree2_checks, random_tree, sumproduct_llr_exact


@pytest.mark.parametrize("seed", range(5))
def test_sumproduct_marginals_exact_on_trees(seed):
    rng = np.random.default_rng(200 + seed)
    H = random_tree(rng, n_checks=int(rng.integers(3, 6)), max_new=2)
    M, N = H.shape
    p = rng.uniform(0.05, 0.4, N)
    row_ptr, col_idx = csr(H)
    sig = rng.integers(0, 2, (3, M)).astype(np.uint8)
    T = 2 * (M + N)
    _, _, _, Lam = soft_dmem(row_ptr, col_idx, p, np.zeros(N), np.ones(T), sig,
                             np.zeros((3, N), np.uint8), grad=False, marginals=True)
    for b in range(3):
        np.testing.assert_allclose(Lam[b], sumproduct_llr_exact(H, p, sig[b]), rtol=1e-9,
                                   atol=1e-9)


def test_soft_degree2_closed_form():
    rng = np.random.default_rng(7)
    N, M, T = 10, 13, 6
    H = random_degree2_checks(rng, N, M)
    row_ptr, col_idx = csr(H)
    p = rng.uniform(0.3, 0.45, N)
    w = np.log((1 - p) / p)
    gam = rng.uniform(-0.2, 0.6, N)
    alpha = rng.uniform(0.3, 0.8, T)
    sig = rng.integers(0, 2, M).astype(np.uint8)
    rows, cols = np.nonzero(H)
    E = rows.size
    Pm = np.zeros((E, E))
    for i in range(M):
        a, b = np.nonzero(rows == i)[0]
        Pm[a, b] = Pm[b, a] = 1
    S = np.diag(np.where(sig[rows] == 1, -1.0, 1.0))
    V = np.zeros((N, E))
    V[cols, np.arange(E)] = 1
    nu, Lam = V.T @ w, w.copy()
    for t in range(T):
        mu = alpha[t] * (S @ Pm @ nu)
        lam = (1 - gam) * w + gam * Lam
        Lam = lam + V @ mu
        nu = V.T @ lam + (V.T @ V - np.eye(E)) @ mu
    _, _, _, got = soft_dmem(row_ptr, col_idx, p, gam, alpha, sig[None, :],
                             np.zeros((1, N), np.uint8), grad=False, marginals=True)
    np.testing.assert_allclose(got[0], Lam, rtol=1e-11, atol=1e-11)


def test_loss_is_mean_bce_of_final_marginals():
    P = code_capacity_dem(BB72, 0.05)
    F = sample_faults(P.p, 3, 6)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    L, _, _, Lam = soft_dmem(P.row_ptr, P.col_idx, P.p, np.full(P.N, 0.125), np.full(8, 0.5),
                             s, F, grad=False, marginals=True)
    q = 1 / (1 + np.exp(Lam))            # P(F_j = 1) = sigmoid(-Lambda_j)
    bce = -(F * np.log(q) + (1 - F) * np.log(1 - q))
    assert abs(L - bce.mean()) < 1e-12 * max(1.0, L)


def test_reverse_pass_matches_central_differences_72_qubit_code():
    """[[72,12,6]] code capacity, 25 iterations, random gamma_j and alpha_t."""
    P = code_capacity_dem(BB72, 0.05)
    F = sample_faults(P.p, 5, 12)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    rng = np.random.default_rng(1)
    gam = rng.uniform(0.0, 0.3, P.N)
    alpha = rng.uniform(0.25, 0.4, 25)   # unsaturated: no product reaches the clamp
    L, gg, ga, _ = soft_dmem(P.row_ptr, P.col_idx, P.p, gam, alpha, s, F)
    h = 1e-6

    def loss(g, a):
        return soft_dmem(P.row_ptr, P.col_idx, P.p, g, a, s, F, grad=False)[0]

    fd_g = np.array([(loss(gam + h * e, alpha) - loss(gam - h * e, alpha)) / (2 * h)
                     for e in np.eye(P.N)])
    fd_a = np.array([(loss(gam, alpha + h * e) - loss(gam, alpha - h * e)) / (2 * h)
                     for e in np.eye(25)])
    assert np.abs(fd_g - gg).max() <= 1e-6 * np.abs(gg).max()
    assert np.abs(fd_a - ga).max() <= 1e-6 * np.abs(ga).max()
