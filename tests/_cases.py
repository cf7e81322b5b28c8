"""Shared test cases: decoding problems, syndromes and helpers to run both sides."""
from __future__ import annotations

import functools

import numpy as np

from workloads import (BB72, BB144, BB288, code_capacity_dem, gamma_table, pack_bits,
                       phenomenological_dem, sample_faults, syndromes_of, unpack_bits)

GAMMA_RANGE = {"bb72": (-0.24, 0.66), "bb144": (-0.24, 0.66), "bb288": (-0.161, 0.815)}


@functools.lru_cache(maxsize=None)
def problem(name: str):
    """Named decoding problems of the workloads (code, rounds, p)."""
    if name == "bb72_cc":
        return code_capacity_dem(BB72, 0.05)
    if name == "bb72_T6":
        return phenomenological_dem(BB72, 6, 0.003)
    if name == "bb144_T12":
        return phenomenological_dem(BB144, 12, 0.003)
    if name == "bb288_T18":
        return phenomenological_dem(BB288, 18, 0.003)
    raise KeyError(name)


def gamma_for(P, R=300, seed=0):
    lo, hi = GAMMA_RANGE[P.meta["code"]]
    return gamma_table(P.N, R, 0.125, lo, hi, seed)


def shots(P, n, seed, first=0):
    F = sample_faults(P.p, seed, n, first_shot=first)
    return F, syndromes_of(P.row_ptr, P.col_idx, F)


def syndrome(P, F):
    return ((F.astype(np.int64) @ P.H.T.astype(np.int64)) % 2).astype(np.uint8)


def gpu_decode(P, gam, sig, cfg, device=0):
    """Decode uint8 syndromes [B, M] with the CUDA library; returns numpy outputs."""
    import torch
    from paper_2511_21660_gb300 import RelayDecoder
    dec = RelayDecoder(P.row_ptr, P.col_idx, P.p, gam, cfg, device)
    try:
        syn = torch.from_numpy(pack_bits(sig).view(np.int64)).cuda(device)
        cor, legs, conv, iters = dec.decode(syn)
        torch.cuda.synchronize()
        return (unpack_bits(cor.cpu().numpy().view(np.uint64), P.N), legs.cpu().numpy(),
                conv.cpu().numpy(), iters.cpu().numpy(), dec.info)
    finally:
        dec.close()


def assert_same_decisions(got, ref, label=""):
    cor, legs, conv, iters = got[:4]
    bad = np.nonzero((cor != ref.corrections).any(1) | (legs != ref.legs)
                     | (conv != ref.converged) | (iters != ref.iters))[0]
    assert bad.size == 0, (f"{label}: {bad.size} shots differ, first {bad[:5]}: "
                           f"legs {legs[bad[:3]]} vs {ref.legs[bad[:3]]}, "
                           f"iters {iters[bad[:3]]} vs {ref.iters[bad[:3]]}")


def logical_failures(P, F, cor, conv):
    res = (F ^ cor).astype(np.int64)
    return ((res @ P.A.T.astype(np.int64)) % 2).any(1) | (conv == 0)
