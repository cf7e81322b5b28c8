"""Pins for the seeded input generators (codes, detector matrices, sampler, gamma table)."""
import json
import os

import numpy as np
import pytest

from workloads import (BB72, BB144, BB288, code_capacity_dem, gamma_table, gf2_nullspace,
                       gf2_rank, pack_bits, phenomenological_dem, sample_faults, splitmix64,
                       syndromes_of, unpack_bits)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("code,rank", [(BB72, 30), (BB144, 66), (BB288, 138)])
def test_bb_code_parameters(code, rank):
    hx, hz = code.hx, code.hz
    assert ((hx.astype(int) @ hz.T.astype(int)) % 2 == 0).all()       # CSS condition
    assert gf2_rank(hx) == rank and gf2_rank(hz) == rank
    assert code.k == 12
    assert set(hx.sum(0)) == {3} and set(hx.sum(1)) == {6}


@pytest.mark.parametrize("code", [BB72, BB144])
def test_x_logicals(code):
    lx = code.x_logicals()
    assert lx.shape == (12, code.n)
    assert ((code.hz.astype(int) @ lx.T.astype(int)) % 2 == 0).all()
    assert gf2_rank(np.vstack([code.hx, lx])) == gf2_rank(code.hx) + 12


def test_detector_matrices_match_paper_row_counts():
    g = json.load(open(os.path.join(GOLDEN, "relay_parameters_appA3.json")))
    P = phenomenological_dem(BB144, 12, 0.003)
    assert P.M == g["detector_rows_gross"]
    P2 = phenomenological_dem(BB288, 18, 0.003)
    assert P2.M == g["detector_rows_two_gross"]


@pytest.mark.parametrize("code,T,shape,E", [(BB72, 6, (252, 720), 1944),
                                            (BB144, 12, (936, 2736), 7344),
                                            (BB288, 18, (2736, 8064), 21600)])
def test_phenomenological_shapes(code, T, shape, E):
    P = phenomenological_dem(code, T, 0.003)
    assert (P.M, P.N) == shape and P.E == E
    assert set(P.H.sum(1).tolist()) == {7, 8}
    assert set(P.H.sum(0).tolist()) == {2, 3}
    # measurement faults only flip detectors of consecutive rounds of one check
    n_data = P.meta["n_data"]
    rows = [np.nonzero(P.H[:, c])[0] for c in range(n_data, P.N)]
    mx = code.hx.shape[0]
    assert all(r[1] - r[0] == mx for r in rows)
    # a data fault in the final (perfect) round still flips its H_X column there
    last = n_data - code.n
    assert (P.H[T * mx:, last:n_data] == code.hx).all()
    # logical action: data columns carry the X-logicals, measurement columns nothing
    assert (P.A[:, n_data:] == 0).all()


def test_dem_logical_action_is_consistent():
    """A residual in ker(H) fails iff its net data part is a logical (not in rowspace H_Z)."""
    P = phenomenological_dem(BB72, 3, 0.003)
    code = BB72
    rng = np.random.default_rng(5)
    ker = gf2_nullspace(P.H)
    rz = gf2_rank(code.hz)
    for _ in range(40):
        r = (rng.integers(0, 2, ker.shape[0]) @ ker) % 2
        net = r[:P.meta["n_data"]].reshape(-1, code.n).sum(0) % 2
        logical = gf2_rank(np.vstack([code.hz, net])) > rz
        assert logical == bool(((P.A.astype(int) @ r) % 2).any())


def test_splitmix64_reference_values():
    # First outputs of SplitMix64 for seeds 0 and 1234567 (Vigna's reference generator).
    assert int(splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    assert int(splitmix64(np.uint64(1234567))) == 6457827717110365317


def test_sampler_is_counter_based_and_calibrated():
    p = np.full(500, 0.01)
    a = sample_faults(p, 3, 64)
    b = sample_faults(p, 3, 16, first_shot=40)
    assert (a[40:56] == b).all()
    assert not (sample_faults(p, 4, 64) == a).all()
    big = sample_faults(np.full(1000, 0.05), 9, 400)
    m = big.mean()
    assert abs(m - 0.05) < 4 * np.sqrt(0.05 * 0.95 / big.size)


def test_syndromes_of_matches_dense_product():
    P = phenomenological_dem(BB72, 2, 0.01)
    F = sample_faults(P.p, 11, 50)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    assert (s == (F.astype(int) @ P.H.T.astype(int)) % 2).all()


def test_pack_bits_layout():
    bits = np.zeros((2, 130), dtype=np.uint8)
    bits[0, 0] = 1
    bits[0, 65] = 1
    bits[1, 129] = 1
    w = pack_bits(bits)
    assert w.shape == (2, 3)
    assert w[0, 0] == 1 and w[0, 1] == 2 and w[1, 2] == 2
    assert (unpack_bits(w, 130) == bits).all()


def test_gamma_table():
    g = gamma_table(100, 7, 0.125, -0.24, 0.66, 2)
    assert g.shape == (8, 100)
    assert (g[0] == 0.125).all()
    assert g[1:].min() >= -0.24 and g[1:].max() <= 0.66
    assert (g.astype(np.float32).astype(np.float64) == g).all()
    assert abs(g[1:].mean() - 0.21) < 0.05
    assert not np.array_equal(g[1], g[2])


def test_code_capacity_problem():
    P = code_capacity_dem(BB72, 0.05)
    assert (P.M, P.N, P.E) == (36, 72, 216)


def test_torch_sampler_is_bit_identical_to_numpy_sampler():
    torch = pytest.importorskip("torch")
    from workloads.torch_sampling import pack_bits_t, sample_faults_t, syndromes_t
    P = phenomenological_dem(BB72, 3, 0.02)
    p = P.p.copy()
    p[:5] = [0.5, 1e-9, 0.3, 0.0031, 0.25]
    F = sample_faults(p, 7, 300, first_shot=1000)
    Ft = sample_faults_t(p, 7, 300, first_shot=1000, chunk=128)
    assert np.array_equal(Ft.numpy(), F)
    s = syndromes_of(P.row_ptr, P.col_idx, F)
    st = syndromes_t(P.H, Ft)
    assert np.array_equal(st.numpy(), s)
    assert np.array_equal(pack_bits_t(st).numpy().view(np.uint64), pack_bits(s))
