"""Parity of the CUDA decoder (through the C ABI) with the CPU oracle.

Hard decisions, convergence, leg and iteration counts are compared bit for bit
with the oracle built in the kernel's precision (float32 arithmetic, with or
without binary16 message storage); messages and marginals of the first
iterations are compared with the FP64 oracle within 1e-4 relative; logical error
rates are compared with the FP64 oracle within 2 sigma.
"""
import numpy as np
import pytest

from oracle.relay import RelayParams, dmem_trace, relay_decode
from workloads import pack_bits

from _cases import (assert_same_decisions, gamma_for, gpu_decode, logical_failures, problem,
                    shots, syndrome)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2511_21660_gb300 import (QLDPC_KERNEL_BASELINE, QLDPC_KERNEL_FUSED,  # noqa: E402
                                    QLDPC_MSG_FP16, QLDPC_MSG_FP32, RelayConfig, RelayDecoder)

PREC = {QLDPC_MSG_FP32: "f32", QLDPC_MSG_FP16: "f16s"}


def _params(cfg: RelayConfig) -> RelayParams:
    return RelayParams(legs_after_first=cfg.legs_after_first, iters_first=cfg.iters_first,
                       iters_later=cfg.iters_later, max_total_iters=cfg.max_total_iters,
                       stop_after_solutions=cfg.stop_after_solutions,
                       warm_start_mode=cfg.warm_start_mode)


CASES = [("bb72_cc", 2000, 0), ("bb72_T6", 600, 2), ("bb144_T12", 600, 1), ("bb288_T18", 120, 2)]


@pytest.mark.parametrize("name,n,seed", CASES)
@pytest.mark.parametrize("prec", [QLDPC_MSG_FP32, QLDPC_MSG_FP16])
def test_fused_matches_mirror_bit_for_bit(name, n, seed, prec):
    P = problem(name)
    F, sig = shots(P, n, seed)
    gam = gamma_for(P, seed=seed)
    cfg = RelayConfig(stop_after_solutions=5, msg_precision=prec, kernel=QLDPC_KERNEL_FUSED)
    got = gpu_decode(P, gam, sig, cfg)
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, _params(cfg), precision=PREC[prec])
    assert_same_decisions(got, ref, f"{name}/{PREC[prec]}")
    ok = got[2] == 1
    assert (syndrome(P, got[0][ok]) == sig[ok]).all()


@pytest.mark.parametrize("warm_mode", [0, 1])
@pytest.mark.parametrize("S", [1, 5])
def test_fused_modes_and_solution_counts(warm_mode, S):
    P = problem("bb72_T6")
    F, sig = shots(P, 400, 5)
    gam = gamma_for(P, seed=5)
    cfg = RelayConfig(stop_after_solutions=S, warm_start_mode=warm_mode)
    got = gpu_decode(P, gam, sig, cfg)
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, _params(cfg), precision="f32")
    assert_same_decisions(got, ref, f"mode{warm_mode}/S{S}")


@pytest.mark.parametrize("name,n", [("bb72_cc", 1000), ("bb144_T12", 300)])
def test_baseline_matches_mirror_bit_for_bit(name, n):
    P = problem(name)
    F, sig = shots(P, n, 3)
    gam = gamma_for(P, seed=3)
    cfg = RelayConfig(stop_after_solutions=5, kernel=QLDPC_KERNEL_BASELINE)
    got = gpu_decode(P, gam, sig, cfg)
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, _params(cfg), precision="f32")
    assert_same_decisions(got, ref, f"baseline/{name}")


def test_hard_shots_with_high_noise():
    """p = 0.03 on the gross code: many legs per shot, some shots never converge."""
    from workloads import BB144, phenomenological_dem
    P = phenomenological_dem(BB144, 12, 0.03)
    P.meta["code"] = "bb144"
    F, sig = shots(P, 48, 9)
    gam = gamma_for(P, seed=9)
    cfg = RelayConfig(stop_after_solutions=1, max_total_iters=3000)
    got = gpu_decode(P, gam, sig, cfg)
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, _params(cfg), precision="f32")
    assert_same_decisions(got, ref, "high-noise")
    assert ref.legs.max() > 3


def test_unsolvable_syndrome_runs_to_the_paper_bound():
    from workloads import gf2_nullspace
    P = problem("bb72_cc")
    y = gf2_nullspace(P.H.T)[0]
    sig = np.zeros((3, P.M), dtype=np.uint8)
    sig[:, np.nonzero(y)[0][0]] = 1
    gam = gamma_for(P)
    for prec in (QLDPC_MSG_FP32, QLDPC_MSG_FP16):
        cor, legs, conv, iters, _ = gpu_decode(P, gam, sig, RelayConfig(msg_precision=prec))
        assert (iters == 80 + 300 * 60).all() and (legs == 301).all() and (conv == 0).all()
        ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, RelayParams(),
                           precision=PREC[prec])
        assert (cor == ref.corrections).all()
    cor, legs, conv, iters, _ = gpu_decode(P, gam, sig, RelayConfig(max_total_iters=1000))
    assert (iters == 1000).all() and (legs == 17).all() and (conv == 0).all()


def test_zero_syndromes_and_empty_batch():
    P = problem("bb144_T12")
    gam = gamma_for(P)
    sig = np.zeros((5, P.M), dtype=np.uint8)
    cor, legs, conv, iters, _ = gpu_decode(P, gam, sig, RelayConfig(stop_after_solutions=5))
    assert cor.sum() == 0 and (iters == 5).all() and (legs == 5).all() and (conv == 1).all()
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig())
    empty = torch.zeros((0, dec.syndrome_words), dtype=torch.int64, device="cuda")
    out = dec.decode(empty)
    torch.cuda.synchronize()
    assert out[0].shape[0] == 0
    dec.close()


def test_irregular_graph_with_degree_one_checks_and_erasures():
    """Ragged sizes, degree-1 checks (empty excluded set), erasures (w = 0), high degrees."""
    rng = np.random.default_rng(11)
    M, N = 45, 101
    H = np.zeros((M, N), dtype=np.uint8)
    for j in range(5, N):
        H[rng.choice(M, int(rng.integers(1, 7)), replace=False), j] = 1
    H[:, 3] = 0
    H[rng.choice(np.arange(1, M), 8, replace=False), 3] = 1   # a fault of degree 8
    H[0, :] = 0
    H[0, 7] = 1                                          # a check of degree 1
    H[1, :] = 0                                          # a check of degree 0
    assert H.sum(0).max() <= 8 and 8 < H.sum(1).max() <= 16
    from workloads import DecodingProblem
    p = rng.uniform(0.01, 0.2, N)
    p[10:14] = 0.5                                       # erasures: w = 0 exactly
    P = DecodingProblem("irregular", H, np.zeros((1, N), np.uint8), p, {"code": "bb72"})
    F = (rng.random((300, N)) < p).astype(np.uint8)
    sig = syndrome(P, F)
    gam = gamma_for(P, R=20, seed=4)
    for prec in (QLDPC_MSG_FP32, QLDPC_MSG_FP16):
        cfg = RelayConfig(legs_after_first=20, stop_after_solutions=3, msg_precision=prec)
        got = gpu_decode(P, gam, sig, cfg)
        assert got[4].max_check_degree > 8 and got[4].max_fault_degree == 8
        ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, _params(cfg),
                           precision=PREC[prec])
        assert_same_decisions(got, ref, f"irregular/{PREC[prec]}")


def _random_graph(rng, M, N, dv_max, n_wide, dc_wide):
    """Random H with fault degrees 1..dv_max, plus n_wide checks of degree in dc_wide."""
    H = np.zeros((M, N), dtype=np.uint8)
    for j in range(N):
        H[rng.choice(M, int(rng.integers(1, dv_max + 1)), replace=False), j] = 1
    for i in rng.choice(M, n_wide, replace=False):
        H[i, :] = 0
        free = np.nonzero(H.sum(0) < dv_max)[0]
        H[i, rng.choice(free, int(rng.integers(*dc_wide)), replace=False)] = 1
    return H


def test_widest_check_family():
    """Checks of degree 17..32 (the widest compiled family), both precisions."""
    rng = np.random.default_rng(21)
    from workloads import DecodingProblem
    H = _random_graph(rng, 150, 300, 4, 6, (17, 33))
    assert 16 < H.sum(1).max() <= 32 and H.sum(0).max() <= 8
    p = rng.uniform(0.01, 0.1, 300)
    P = DecodingProblem("wide", H, np.zeros((1, 300), np.uint8), p, {"code": "bb72"})
    F = (rng.random((200, 300)) < p).astype(np.uint8)
    sig = syndrome(P, F)
    gam = gamma_for(P, R=20, seed=5)
    for prec in (QLDPC_MSG_FP32, QLDPC_MSG_FP16):
        cfg = RelayConfig(legs_after_first=20, stop_after_solutions=3, msg_precision=prec)
        got = gpu_decode(P, gam, sig, cfg)
        assert got[4].max_check_degree > 16
        ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, _params(cfg),
                           precision=PREC[prec])
        assert_same_decisions(got, ref, f"wide/{PREC[prec]}")


@pytest.mark.parametrize("prec", [QLDPC_MSG_FP32, QLDPC_MSG_FP16])
def test_largest_graph_the_default_family_holds(prec):
    """N = 12,000 faults: the largest shape of the degree-8/4 family (512 x 32); its
    float32 message array (144 KB) and priors fill most of a block's shared memory."""
    rng = np.random.default_rng(22)
    from workloads import DecodingProblem
    M, N = 4500, 12000
    sockets = rng.permutation(np.repeat(np.arange(M), 8)).reshape(N, 3)  # 8 per check, 3 per fault
    H = np.zeros((M, N), dtype=np.uint8)
    H[sockets.ravel(), np.repeat(np.arange(N), 3)] = 1                 # repeated pairs merge
    p = np.full(N, 0.002)
    P = DecodingProblem("large", H, np.zeros((1, N), np.uint8), p, {"code": "bb72"})
    F = (rng.random((40, N)) < p).astype(np.uint8)
    sig = syndrome(P, F)
    gam = gamma_for(P, R=10, seed=6)
    cfg = RelayConfig(legs_after_first=10, stop_after_solutions=2, msg_precision=prec)
    got = gpu_decode(P, gam, sig, cfg)
    assert got[4].block_threads == 512 and got[4].max_check_degree <= 8
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, _params(cfg), precision=PREC[prec])
    assert_same_decisions(got, ref, "largest")


@pytest.mark.parametrize("prec", [QLDPC_MSG_FP32, QLDPC_MSG_FP16])
def test_small_saturation_bound_clamps_like_the_oracle(prec):
    """llr_clip = 12: messages and marginals saturate all the time (R11); both precisions
    take the general clamp path (binary16's saturating store applies only at 65504)."""
    P = problem("bb72_T6")
    F, sig = shots(P, 400, 9)
    gam = gamma_for(P, seed=9)
    cfg = RelayConfig(stop_after_solutions=5, msg_precision=prec, llr_clip=12.0)
    got = gpu_decode(P, gam, sig, cfg)
    prm = _params(cfg)
    prm.clip = 12.0
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, prm, precision=PREC[prec])
    assert_same_decisions(got, ref, f"clip12/{PREC[prec]}")


def test_host_buffer_entry_point_matches_device_entry_point():
    P = problem("bb144_T12")
    F, sig = shots(P, 500, 6)
    gam = gamma_for(P, seed=6)
    cfg = RelayConfig(stop_after_solutions=5)
    dev = gpu_decode(P, gam, sig, cfg)
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, cfg)
    cor, legs, conv, iters = dec.decode_host(pack_bits(sig))
    dec.close()
    from workloads import unpack_bits
    assert (unpack_bits(cor, P.N) == dev[0]).all()
    assert (legs == dev[1]).all() and (conv == dev[2]).all() and (iters == dev[3]).all()


@pytest.mark.parametrize("name", ["bb72_cc", "bb144_T12"])
def test_host_buffer_entry_point_matches_device_entry_point_on_a_large_batch(name):
    """A batch of 16 grids of shots and a ragged remainder through the host buffers."""
    P = problem(name)
    gam = gamma_for(P, seed=7)
    cfg = RelayConfig(stop_after_solutions=5)
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, cfg)
    n = 16 * dec.info.grid_blocks + 37
    F, sig = shots(P, n, 7)
    cor, legs, conv, iters = dec.decode_host(pack_bits(sig))
    dec.close()
    dev = gpu_decode(P, gam, sig, cfg)
    from workloads import unpack_bits
    assert (unpack_bits(cor, P.N) == dev[0]).all()
    assert (legs == dev[1]).all() and (conv == dev[2]).all() and (iters == dev[3]).all()


@pytest.mark.parametrize("prec", [QLDPC_MSG_FP32, QLDPC_MSG_FP16])
def test_first_iterations_match_fp64_oracle(prec):
    """Messages and marginals over the first 10 iterations (relative error in LLR units)."""
    P = problem("bb144_T12")
    F, sig = shots(P, 32, 8)
    gam = gamma_for(P)
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(msg_precision=prec))
    marg, nu, mu = dec.trace_first_leg(torch.from_numpy(pack_bits(sig).view(np.int64)).cuda(), 10)
    torch.cuda.synchronize()
    dec.close()
    marg = marg.cpu().numpy().transpose(1, 0, 2)
    nu = nu.cpu().numpy().transpose(1, 0, 2)
    mu = mu.cpu().numpy().transpose(1, 0, 2)
    L64, nu64, mu64 = dmem_trace(P.row_ptr, P.col_idx, P.p, gam[0], sig, 10,
                                 clip=65504.0 if prec == QLDPC_MSG_FP16 else 1e30)
    # float32: the 1e-4 target.  binary16 storage: each stored message is rounded with
    # unit roundoff 2^-11 = 4.9e-4, and over 10 iterations a fault sums up to three
    # such messages per iteration, so the bound is 10 * 3 * 2^-11 = 1.5e-2.
    tol = 1e-4 if prec == QLDPC_MSG_FP32 else 10 * 3 * 2.0 ** -11
    for a, b, what in ((marg, L64, "Lambda"), (nu, nu64, "nu"), (mu, mu64, "mu")):
        err = np.abs(a - b) / np.maximum(1.0, np.abs(b))
        assert err.max() <= tol, (what, float(err.max()))
    # the mirror in the kernel's own precision is matched exactly
    L32, nu32, mu32 = dmem_trace(P.row_ptr, P.col_idx, P.p, gam[0], sig, 10, precision=PREC[prec])
    assert (marg == L32).all() and (nu == nu32).all() and (mu == mu32).all()


def test_logical_error_rate_matches_fp64_oracle_code_capacity():
    """[[72,12,6]] code capacity, p = 0.05, 10,000 shots, seed 0, S = 5."""
    P = problem("bb72_cc")
    F, sig = shots(P, 10000, 0)
    gam = gamma_for(P, seed=0)
    cfg = RelayConfig(stop_after_solutions=5)
    got = gpu_decode(P, gam, sig, cfg)
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig, _params(cfg), precision="f64")
    f_gpu = logical_failures(P, F, got[0], got[2])
    f_ora = logical_failures(P, F, ref.corrections, ref.converged)
    n = F.shape[0]
    pbar = (f_gpu.mean() + f_ora.mean()) / 2
    sigma = np.sqrt(max(pbar * (1 - pbar), 1.0 / n) * 2.0 / n)
    assert abs(f_gpu.mean() - f_ora.mean()) <= 2 * sigma, (f_gpu.mean(), f_ora.mean())
    ok = got[2] == 1
    assert (syndrome(P, got[0][ok]) == sig[ok]).all()


_FULL = {}


def _full_size_inputs():
    if not _FULL:
        P = problem("bb144_T12")
        F, sig = shots(P, 100000, 1)
        _FULL["P"], _FULL["sig"], _FULL["gam"] = P, sig, gamma_for(P, seed=1)
    return _FULL["P"], _FULL["sig"], _FULL["gam"]


# every block shape the benchmark's autotuner chooses from, in both message precisions
@pytest.mark.parametrize("prec,bt",
                         [(QLDPC_MSG_FP32, b) for b in (256, 384, 512, 640, 768, 1024)]
                         + [(QLDPC_MSG_FP16, b) for b in (384, 512)])
def test_full_size_gross_batch_sampled_parity(prec, bt):
    """10^5 gross-code shots in the benchmark's launch configurations."""
    P, sig, gam = _full_size_inputs()
    cfg = RelayConfig(stop_after_solutions=5, msg_precision=prec, block_threads=bt)
    cor, legs, conv, iters, info = gpu_decode(P, gam, sig, cfg)
    assert info.block_threads == bt
    ok = conv == 1
    from workloads import syndromes_of
    assert (syndromes_of(P.row_ptr, P.col_idx, cor[ok]) == sig[ok]).all()
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(sig.shape[0], 300, replace=False))
    pick = np.union1d(pick, np.argsort(iters)[-20:])     # include the slowest shots
    key = ("ref", PREC[prec], tuple(pick[:3]))
    if key not in _FULL:
        _FULL[key] = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig[pick], _params(cfg),
                                  precision=PREC[prec])
    assert_same_decisions((cor[pick], legs[pick], conv[pick], iters[pick]), _FULL[key],
                          f"full-size {bt}")
