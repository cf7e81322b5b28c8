"""Seeded, counter-based randomness for the synthetic workloads.

Every random number is a pure function of (seed, stream, index), so any shard or
subset of a workload can be regenerated on its own:

    x = (seed << 40) | (stream << 16) | index          (stream < 2^24, index < 2^16)
    z = splitmix64(x)                                  (first output of SplitMix64 seeded with x)
    u = (z >> 11) * 2^-53                              (uniform double in [0, 1))

SplitMix64 is the generator of Steele, Lea and Flood (OOPSLA 2014): add the
golden-ratio increment 0x9E3779B97F4A7C15, then apply the two xor-shift-multiply
rounds with 0xBF58476D1CE4E5B9 and 0x94D049BB133111EB and a final xor-shift.

Faults: fault j of shot s fires iff u(seed, s, j) < p_j.
Memory strengths (the random draws Relay makes for legs r >= 1, Sec. 2.3 "Relay
chaining" and App. A.3): gamma[r, j] = lo + (hi - lo) * u(seed, r, j), rounded to
float32, so that every consumer (FP64 oracle, FP32 kernels) sees identical values.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x) -> np.ndarray:
    """First SplitMix64 output for state(s) x (uint64, wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, streams, n_index: int) -> np.ndarray:
    """u[s, j] in [0,1) for stream ids ``streams`` (1-D) and indices 0..n_index-1."""
    if n_index > (1 << 16):
        raise ValueError("index space is 16 bits")
    streams = np.asarray(streams, dtype=np.uint64)
    if streams.size and int(streams.max()) >= (1 << 24):
        raise ValueError("stream space is 24 bits")
    x = ((np.uint64(seed) << np.uint64(40)) | (streams[:, None] << np.uint64(16))
         | np.arange(n_index, dtype=np.uint64)[None, :])
    z = splitmix64(x)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sample_faults(p: np.ndarray, seed: int, n_shots: int, first_shot: int = 0,
                  chunk: int = 8192) -> np.ndarray:
    """Fault bitstrings F[s, j] = [u(seed, first_shot + s, j) < p_j] as uint8 [n_shots, N]."""
    p = np.asarray(p, dtype=np.float64)
    out = np.empty((n_shots, p.size), dtype=np.uint8)
    for s0 in range(0, n_shots, chunk):
        s1 = min(n_shots, s0 + chunk)
        u = uniform01(seed, np.arange(first_shot + s0, first_shot + s1), p.size)
        out[s0:s1] = u < p[None, :]
    return out


def syndromes_of(row_ptr: np.ndarray, col_idx: np.ndarray, F: np.ndarray,
                 chunk: int = 8192) -> np.ndarray:
    """sigma = H F mod 2 for each row of F (uint8 [B, N]) -> uint8 [B, M]."""
    import scipy.sparse as sp
    M = row_ptr.size - 1
    N = F.shape[1]
    H = sp.csr_matrix((np.ones(col_idx.size, dtype=np.int32), col_idx, row_ptr), shape=(M, N))
    out = np.empty((F.shape[0], M), dtype=np.uint8)
    for s0 in range(0, F.shape[0], chunk):
        s1 = min(F.shape[0], s0 + chunk)
        out[s0:s1] = (np.asarray((H @ F[s0:s1].T.astype(np.int32)).T) & 1).astype(np.uint8)
    return out


def gamma_table(n_vars: int, legs_after_first: int, gamma0: float, lo: float, hi: float,
                seed: int) -> np.ndarray:
    """Memory strengths Gamma[r, j], r = 0..R: row 0 is gamma0, rows r>=1 are U[lo, hi].

    Values are float32-representable and returned as float64.
    """
    g = np.empty((legs_after_first + 1, n_vars), dtype=np.float64)
    g[0] = np.float64(np.float32(gamma0))
    if legs_after_first > 0:
        u = uniform01(seed, np.arange(1, legs_after_first + 1), n_vars)
        g[1:] = (lo + (hi - lo) * u).astype(np.float32).astype(np.float64)
    return g


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """uint8 0/1 [B, n] -> uint64 [B, ceil(n/64)]; bit k of word w is entry 64w+k."""
    bits = np.asarray(bits, dtype=np.uint8)
    B, n = bits.shape
    words = (n + 63) // 64
    padded = np.zeros((B, words * 64), dtype=np.uint8)
    padded[:, :n] = bits
    by = np.packbits(padded, axis=1, bitorder="little")
    return np.ascontiguousarray(by).view("<u8").astype(np.uint64).reshape(B, words)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    """Inverse of pack_bits: uint64 [B, W] -> uint8 [B, n]."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64).astype("<u8"))
    by = w.view(np.uint8).reshape(w.shape[0], -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :n].copy()
