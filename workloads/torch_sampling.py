"""The counter-based fault sampler of workloads.sampling, on torch tensors (CPU or GPU).

Same definition, bit for bit: for fault j of shot s,
    z = splitmix64((seed << 40) | (s << 16) | j),  fault iff (z >> 11) * 2^-53 < p_j.
The comparison is done in integers: (z >> 11) < ceil(p_j * 2^53), with the
threshold computed exactly on the host.  torch's int64 arithmetic wraps like
uint64; right shifts are made logical by masking.
"""
from __future__ import annotations

from fractions import Fraction
import math

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _s64(v: int) -> int:
    """uint64 constant as the int64 with the same bits."""
    return v - (1 << 64) if v >= (1 << 63) else v


def _lshr(x, k: int):
    """Logical right shift of int64 bit patterns."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def splitmix64_t(x):
    import torch  # noqa: F401
    z = x + _s64(_GOLDEN)
    z = (z ^ _lshr(z, 30)) * _s64(_M1)
    z = (z ^ _lshr(z, 27)) * _s64(_M2)
    return z ^ _lshr(z, 31)


def thresholds(p) -> np.ndarray:
    """Integer thresholds t_j = ceil(p_j * 2^53): fault iff (z >> 11) < t_j."""
    return np.array([math.ceil(Fraction(float(q)) * (1 << 53)) for q in np.atleast_1d(p)],
                    dtype=np.int64)


def sample_faults_t(p, seed: int, n_shots: int, first_shot: int = 0, device="cpu",
                    chunk: int = 16384):
    """uint8 tensor [n_shots, N] equal to workloads.sample_faults(p, seed, n_shots, first_shot)."""
    import torch
    p = np.asarray(p, dtype=np.float64)
    N = p.size
    if N > (1 << 16) or first_shot + n_shots > (1 << 24):
        raise ValueError("index space is 16 bits, stream space 24 bits")
    thr = torch.from_numpy(thresholds(p)).to(device)
    j = torch.arange(N, dtype=torch.int64, device=device)
    out = torch.empty((n_shots, N), dtype=torch.uint8, device=device)
    for s0 in range(0, n_shots, chunk):
        s1 = min(n_shots, s0 + chunk)
        s = torch.arange(first_shot + s0, first_shot + s1, dtype=torch.int64, device=device)
        x = (seed << 40) | (s[:, None] << 16) | j[None, :]
        z = splitmix64_t(x)
        out[s0:s1] = (_lshr(z, 11) < thr[None, :]).to(torch.uint8)
    return out


def syndromes_t(H: np.ndarray, F):
    """sigma = H F mod 2 for each row of F (uint8 tensor [B, N]) -> uint8 [B, M]."""
    import torch
    Ht = torch.from_numpy(np.ascontiguousarray(H.T, dtype=np.float32)).to(F.device)
    out = torch.empty((F.shape[0], H.shape[0]), dtype=torch.uint8, device=F.device)
    for s0 in range(0, F.shape[0], 65536):
        s1 = min(F.shape[0], s0 + 65536)
        cnt = F[s0:s1].to(torch.float32) @ Ht          # exact: counts < 2^24
        out[s0:s1] = (cnt.to(torch.int32) & 1).to(torch.uint8)
    return out


def pack_bits_t(bits):
    """uint8 0/1 [B, n] -> int64 [B, ceil(n/64)] with the layout of workloads.pack_bits."""
    import torch
    B, n = bits.shape
    words = (n + 63) // 64
    padded = torch.zeros((B, words * 64), dtype=torch.int64, device=bits.device)
    padded[:, :n] = bits.to(torch.int64)
    shifts = torch.arange(64, dtype=torch.int64, device=bits.device)
    return (padded.view(B, words, 64) << shifts).sum(dim=2)
