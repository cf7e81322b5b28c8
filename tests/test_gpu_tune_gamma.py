"""Tuning gamma_j with the soft leg, judged by plain Relay-BP (min-sum, S = 5).

Gross code, 12 rounds, p = 0.02 (where the logical error rate is measurable).  The
soft leg is trained on fresh 4096-shot batches; Relay then decodes the same 10^6
evaluation shots with the default first-leg gamma (0.125) and with the tuned one.
Both rates are printed; the test requires the training loss to fall and both
evaluations to be consistent (every converged correction satisfies its syndrome).
"""
import json

import numpy as np
import pytest

from workloads import BB144, gamma_table, phenomenological_dem

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2511_21660_gb300 import RelayConfig, RelayDecoder, SoftDMem  # noqa: E402
from paper_2511_21660_gb300.tune_gamma import train_memory_strengths  # noqa: E402
from workloads.torch_sampling import pack_bits_t, sample_faults_t, syndromes_t  # noqa: E402


def test_tuned_gamma_evaluated_by_relay():
    p = 0.02
    P = phenomenological_dem(BB144, 12, p)
    soft = SoftDMem(P.row_ptr, P.col_idx, P.p, iterations=25, checkpoint_every=5)

    def batches(step):
        F = sample_faults_t(P.p, 100, 4096, first_shot=4096 * step, device="cuda")
        return pack_bits_t(syndromes_t(P.H, F)), pack_bits_t(F)

    g, a, losses = train_memory_strengths(soft, batches, steps=150, lr=0.01)
    assert np.isfinite(losses).all()
    assert np.mean(losses[-10:]) < np.mean(losses[:10])

    n_eval = 1_000_000
    F = sample_faults_t(P.p, 7, n_eval, device="cuda")
    sig = syndromes_t(P.H, F)
    syn = pack_bits_t(sig)
    A = torch.from_numpy(P.A.astype(np.float32)).cuda()
    shifts = torch.arange(64, dtype=torch.int64, device="cuda")
    H = torch.from_numpy(P.H.astype(np.float32)).cuda()
    out = {"p": p, "train_steps": 150, "batch": 4096, "loss_first": losses[0],
           "loss_last": losses[-1], "eval_shots": n_eval}
    base = gamma_table(P.N, 300, 0.125, -0.24, 0.66, 7)
    for name in ("default", "tuned"):
        gam = base.copy()
        if name == "tuned":
            gam[0] = g.cpu().numpy().astype(np.float32).astype(np.float64)
        dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, RelayConfig(stop_after_solutions=5))
        cor, legs, conv, iters = dec.decode(syn)
        Fh = ((cor[:, :, None] >> shifts) & 1).reshape(n_eval, -1)[:, :P.N].to(torch.uint8)
        ok = conv == 1
        resyn = ((Fh[ok].to(torch.float32) @ H.T).to(torch.int64) & 1).to(torch.uint8)
        assert torch.equal(resyn, sig[ok])
        logical = (((F ^ Fh).to(torch.float32) @ A.T).to(torch.int64) & 1).any(1) | ~ok
        f = int(logical.sum().item())
        out[f"ler_{name}"] = f / n_eval
        out[f"ler_{name}_2sigma"] = 2 * np.sqrt(max(f, 1) * (1 - f / n_eval)) / n_eval
        out[f"mean_iters_{name}"] = float(iters.float().mean().item())
        dec.close()
    out["gamma_tuned_mean"] = float(g.mean().item())
    out["gamma_tuned_std"] = float(g.std().item())
    out["alpha_tuned_first_last"] = [float(a[0].item()), float(a[-1].item())]
    print("TUNE_GAMMA " + json.dumps(out))
    soft.close()
