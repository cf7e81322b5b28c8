"""Tune the per-fault memory strengths gamma_j (and the per-iteration scales alpha_t)
by gradient descent on the soft DMem-BP loss (the differentiable leg of the library).

The trained gamma_j are meant for Relay's first leg (row 0 of the gamma table); the
decoder that judges them is plain Relay-BP (min-sum), run separately.
"""
from __future__ import annotations

from typing import Callable, Iterable

from .qldpc import SoftDMem, soft_dmem_loss


def train_memory_strengths(soft: SoftDMem, batches: Callable[[int], tuple], steps: int,
                           gamma0: float = 0.125, alpha0: float = 1.0, lr: float = 0.01,
                           clamp: Iterable[float] = (-1.0, 1.0), log_every: int = 0):
    """Adam on (gamma, alpha).

    batches(step) -> (syndromes, faults): int64 CUDA tensors of bit-packed words
    [B, ceil(M/64)] and [B, ceil(N/64)].  gamma is kept inside `clamp` after every
    step.  Returns (gamma [N], alpha [T], list of losses), CUDA tensors of soft.dtype.
    """
    import torch
    dev = torch.device("cuda", soft.device)
    g = torch.full((soft.N,), gamma0, dtype=soft.dtype, device=dev, requires_grad=True)
    a = torch.full((soft.T,), alpha0, dtype=soft.dtype, device=dev, requires_grad=True)
    opt = torch.optim.Adam([g, a], lr=lr)
    lo, hi = clamp
    losses = []
    for step in range(steps):
        syn, flt = batches(step)
        opt.zero_grad()
        loss = soft_dmem_loss(soft, syn, flt, g, a)
        loss.backward()
        opt.step()
        with torch.no_grad():
            g.clamp_(lo, hi)
        losses.append(float(loss.item()))
        if log_every and step % log_every == 0:
            print(f"step {step}: loss {losses[-1]:.6f}")
    return g.detach(), a.detach(), losses
