"""Tail continuation of the fused decode: long shots move at a leg boundary to a second
launch with one 1024-thread block per SM.  A leg boundary holds Relay's whole state, so
the results must equal the single-launch decode's bit for bit, whether a shot is moved,
resumed after many more legs, or kept in the first launch because the records ran out;
and the oracle mirror agrees on sampled shots."""
import numpy as np
import pytest

from oracle.relay import RelayParams, relay_decode
from workloads import BB144, phenomenological_dem

from _cases import assert_same_decisions, gamma_for, gpu_decode, problem, shots

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
from paper_2511_21660_gb300 import QLDPC_MSG_FP16, QLDPC_MSG_FP32, RelayConfig  # noqa: E402

PREC = {QLDPC_MSG_FP32: "f32", QLDPC_MSG_FP16: "f16s"}


def _hard(n, seed):
    P = phenomenological_dem(BB144, 12, 0.02)
    P.meta["code"] = "bb144"
    F, sig = shots(P, n, seed)
    return P, sig, gamma_for(P, seed=seed)


def _same(a, b):
    for x, y, what in zip(a[:4], b[:4], ("corrections", "legs", "converged", "iters")):
        assert np.array_equal(x, y), what


@pytest.mark.parametrize("prec", [QLDPC_MSG_FP32, QLDPC_MSG_FP16])
def test_continuation_equals_the_single_launch_on_hard_shots(prec):
    """p = 0.02 gross shots: with the default cut (T_1 + 8 T_r = 560 iterations) the
    shots that never converge run their 301 legs through the second launch."""
    P, sig, gam = _hard(4000, 31)
    on = gpu_decode(P, gam, sig, RelayConfig(stop_after_solutions=5, msg_precision=prec))
    off = gpu_decode(P, gam, sig, RelayConfig(stop_after_solutions=5, msg_precision=prec,
                                              tail_cut_iters=-1))
    info = on[4]
    assert info.tail_cut_iters == 80 + 8 * 60 and info.tail_block_threads == 1024
    assert info.tail_records == 4 * info.num_sms and off[4].tail_cut_iters == -1
    assert (on[3] > 560).sum() >= 3             # shots that went through the second launch
    _same(on, off)
    long_ = np.nonzero(on[3] > 560)[0][:6]
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig[long_],
                       RelayParams(stop_after_solutions=5), precision=PREC[prec])
    assert_same_decisions(tuple(x[long_] for x in on[:4]), ref, "continued shots")


@pytest.mark.parametrize("prec", [QLDPC_MSG_FP32, QLDPC_MSG_FP16])
def test_more_candidates_than_records_and_every_leg_boundary(prec):
    """tail_cut_iters = 1: every shot with a second leg is a candidate at its first leg
    end; the first 4 per SM are moved, the others finish in the first launch."""
    P = problem("bb72_T6")
    F, sig = shots(P, 3000, 32)
    gam = gamma_for(P, seed=32)
    cfg = dict(stop_after_solutions=5, msg_precision=prec)
    on = gpu_decode(P, gam, sig, RelayConfig(tail_cut_iters=1, **cfg))
    off = gpu_decode(P, gam, sig, RelayConfig(tail_cut_iters=-1, **cfg))
    assert (on[1] > 1).sum() > on[4].tail_records   # more candidates than records
    _same(on, off)
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, sig[:400], RelayParams(**{
        "stop_after_solutions": 5}), precision=PREC[prec])
    assert_same_decisions(tuple(x[:400] for x in on[:4]), ref, "cut 1")


def test_continuation_with_an_iteration_budget_and_warm_mode_1():
    P, sig, gam = _hard(1500, 33)
    for cfg in (dict(max_total_iters=3000), dict(warm_start_mode=1), dict(stop_after_solutions=1)):
        base = dict(stop_after_solutions=5)
        base.update(cfg)
        on = gpu_decode(P, gam, sig, RelayConfig(tail_cut_iters=100, **base))
        off = gpu_decode(P, gam, sig, RelayConfig(tail_cut_iters=-1, **base))
        _same(on, off)
