"""Precision study on the gross code, 12 rounds: binary16 message storage with float32
sums vs float32 messages vs the FP64 oracle, at p = 0.001 .. 0.004 and, where logical
failures become measurable, p = 0.015 .. 0.025.

Per p: 10^6 shots decoded on the GPU in both precisions; the FP64 oracle decodes the
first 20,000 of them.  The logical error rate of each GPU precision must agree with the
oracle's within 2 sigma on the common shots; paired shot by shot (McNemar), the shots
that only float32 or only FP64 fails must balance within 3 sigma, which has far more
power than comparing the two rates when most failures are shared (binary16's counts are
reported); FP16 against FP32 over all 10^6 shots is reported.  The messages of the first 10 iterations are compared with FP64 (relative
error in LLR units).  Results are printed as one JSON line per p.
"""
import json

import numpy as np
import pytest

from oracle.relay import RelayParams, dmem_trace, relay_decode
from workloads import BB144, gamma_table, phenomenological_dem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2511_21660_gb300 import (QLDPC_MSG_FP16, QLDPC_MSG_FP32, RelayConfig,  # noqa: E402
                                    RelayDecoder)
from workloads.torch_sampling import pack_bits_t, sample_faults_t, syndromes_t  # noqa: E402

N_GPU = 1_000_000
N_ORACLE = 20_000
N_MESSAGES = 256   # shots whose first 10 iterations are compared message by message


def _two_sample_ok(f1, n1, f2, n2):
    p1, p2 = f1 / n1, f2 / n2
    pb = (f1 + f2) / (n1 + n2)
    sigma = np.sqrt(max(pb * (1 - pb), 1.0 / (n1 + n2)) * (1 / n1 + 1 / n2))
    return abs(p1 - p2) <= 2 * sigma, p1, p2, sigma


def _failures(A, F, cor_words, conv, N):
    """converged == 0 or A (F + F_hat) != 0, on the GPU."""
    shifts = torch.arange(64, dtype=torch.int64, device=F.device)
    Fh = ((cor_words[:, :, None] >> shifts) & 1).reshape(F.shape[0], -1)[:, :N].to(torch.uint8)
    res = (F ^ Fh).to(torch.float32)
    logical = (res @ A.T).to(torch.int64) & 1
    return (logical.any(dim=1) | (conv == 0)).to(torch.int64)


# p = 0.001 .. 0.004 is the configured range; at these rates the phenomenological gross
# model shows no failure in 10^6 shots, so 0.015 .. 0.025 are added to compare rates
# that are measurable.
@pytest.mark.parametrize("p,seed", [(0.001, 10), (0.002, 11), (0.003, 12), (0.004, 13),
                                    (0.015, 14), (0.02, 15), (0.025, 16)])
def test_logical_error_rate_and_message_error_by_precision(p, seed):
    P = phenomenological_dem(BB144, 12, p)
    gam = gamma_table(P.N, 300, 0.125, -0.24, 0.66, seed)
    F = sample_faults_t(P.p, seed, N_GPU, device="cuda")
    sig = syndromes_t(P.H, F)
    syn = pack_bits_t(sig)
    A = torch.from_numpy(P.A.astype(np.float32)).cuda()
    fails = {}
    for name, prec in (("fp16", QLDPC_MSG_FP16), ("fp32", QLDPC_MSG_FP32)):
        dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam,
                           RelayConfig(stop_after_solutions=5, msg_precision=prec))
        cor, legs, conv, iters = dec.decode(syn)
        fails[name] = _failures(A, F, cor, conv, P.N)
        dec.close()
    torch.cuda.synchronize()
    s_host = sig[:N_ORACLE].cpu().numpy()
    F_host = F[:N_ORACLE].cpu().numpy()
    ref = relay_decode(P.row_ptr, P.col_idx, P.p, gam, s_host, RelayParams(stop_after_solutions=5))
    res = (F_host ^ ref.corrections).astype(np.int64)
    fail_ora = (((res @ P.A.T.astype(np.int64)) % 2).any(1) | (ref.converged == 0))
    f_ora = int(fail_ora.sum())
    line = {"p": p, "shots_gpu": N_GPU, "shots_oracle": N_ORACLE}
    for name in ("fp16", "fp32"):
        f_all = int(fails[name].sum())
        sub = fails[name][:N_ORACLE].cpu().numpy().astype(bool)
        f_sub = int(sub.sum())
        ok, p_gpu, p_ora, sg = _two_sample_ok(f_sub, N_ORACLE, f_ora, N_ORACLE)
        assert ok, (name, p, f_sub, f_ora)
        # paired on the same shots (McNemar): the shots that only the GPU precision or
        # only FP64 fails.  float32 must balance within 3 sigma, sqrt(b + c); binary16
        # storage is reported (its logical error rate is measurably higher at large p)
        only_gpu, only_ora = int((sub & ~fail_ora).sum()), int((~sub & fail_ora).sum())
        if name == "fp32":
            assert abs(only_gpu - only_ora) <= 3 * np.sqrt(max(only_gpu + only_ora, 1)), \
                (name, p, only_gpu, only_ora)
        line[f"discordant_{name}_vs_fp64"] = [only_gpu, only_ora]
        line[f"ler_{name}"] = f_all / N_GPU
        line[f"ler_{name}_2sigma"] = 2 * np.sqrt(max(f_all, 1) * (1 - f_all / N_GPU)) / N_GPU
        line[f"failures_{name}_on_oracle_shots"] = f_sub
    line["ler_fp64_oracle"] = f_ora / N_ORACLE
    line["failures_fp64_oracle"] = f_ora
    # FP16 against FP32 on all shots is reported, not required (the target is agreement
    # with the FP64 oracle, checked above on the oracle's shots)
    ok, *_ = _two_sample_ok(int(fails["fp16"].sum()), N_GPU, int(fails["fp32"].sum()), N_GPU)
    line["fp16_vs_fp32_within_2sigma_on_all_shots"] = bool(ok)
    # messages of the first 10 iterations of the first leg, N_MESSAGES shots
    for name, prec, clip in (("fp16", QLDPC_MSG_FP16, 65504.0), ("fp32", QLDPC_MSG_FP32, 1e30)):
        L64, nu64, _ = dmem_trace(P.row_ptr, P.col_idx, P.p, gam[0], s_host[:N_MESSAGES], 10,
                                  clip=clip)
        dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(msg_precision=prec))
        marg, nu, _ = dec.trace_first_leg(syn[:N_MESSAGES].contiguous(), 10)
        torch.cuda.synchronize()
        dec.close()
        nu = nu.cpu().numpy().transpose(1, 0, 2)
        err = np.abs(nu - nu64) / np.maximum(1.0, np.abs(nu64))
        line[f"max_message_error_{name}_t10"] = float(err.max())
        line[f"p999_message_error_{name}_t10"] = float(np.quantile(err, 0.999))
        del nu, nu64, err
    line["message_error_shots"] = N_MESSAGES
    assert line["max_message_error_fp32_t10"] <= 1e-4
    print("PRECISION_STUDY " + json.dumps(line))
