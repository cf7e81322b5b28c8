"""ctypes front end of the C Relay-BP oracle (TEST INFRASTRUCTURE ONLY).

Only tests, the smoke check and the benchmark's CPU-baseline leg may import this
module.  It follows paper Sec. 2.3 ("Relay decoding") and App. A.3 step by step;
the readings where the paper is silent are listed in relay_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_P = ctypes.c_void_p
_LIBS: dict = {}


def _lib(kind: str, variant: str):
    key = (kind, variant)
    if key not in _LIBS:
        path = _build.lib_path(kind, variant)
        if not os.path.exists(path):
            _build.build()
        lib = ctypes.CDLL(path)
        if kind == "relay":
            lib.oracle_relay_decode.restype = ctypes.c_int
            lib.oracle_relay_decode.argtypes = [
                ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32,
                ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                _P, ctypes.c_int64, _P, _P, _P, _P, _P, ctypes.c_int32]
            lib.oracle_dmem_trace.restype = ctypes.c_int
            lib.oracle_dmem_trace.argtypes = [
                ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_double, _P,
                ctypes.c_int64, ctypes.c_int32, _P, _P, _P, ctypes.c_int32]
        _LIBS[key] = lib
    return _LIBS[key]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class RelayParams:
    """Relay hyper-parameters (App. A.3 defaults: T_1=80, T_r=60, R=300, S=1)."""
    legs_after_first: int = 300
    iters_first: int = 80
    iters_later: int = 60
    max_total_iters: int = 0
    stop_after_solutions: int = 1
    warm_start_mode: int = 0
    clip: float = 0.0   # <= 0: 65504 for binary16 message storage, else 1e30


@dataclass
class RelayResult:
    corrections: np.ndarray   # uint8 [B, N]
    legs: np.ndarray          # int32 [B]
    converged: np.ndarray     # uint8 [B]
    iters: np.ndarray         # int64 [B]
    final_marginals: np.ndarray = None   # float64 [B, N] when requested


def default_clip(precision: str) -> float:
    """Saturation bound of messages and marginals: the binary16 maximum when
    messages are stored in binary16, else 1e30 (never reached in practice)."""
    return 65504.0 if precision == "f16s" else 1e30


def _csr(row_ptr, col_idx):
    return (np.ascontiguousarray(row_ptr, dtype=np.int32),
            np.ascontiguousarray(col_idx, dtype=np.int32))


def relay_decode(row_ptr, col_idx, priors, gamma, sigma, params: RelayParams,
                 precision: str = "f64", nthreads: int = 0,
                 want_marginals: bool = False) -> RelayResult:
    """Decode syndromes sigma (uint8 [B, M]) with Relay.

    precision: "f64" (the oracle), "f32" (single-precision mirror) or "f16s"
    (single precision with binary16 message storage); "f64_O3" is the FP64 oracle
    compiled at -O3 (same values, the benchmark's timed CPU baseline).
    nthreads: OpenMP threads over shots (0 = all host cores).
    """
    row_ptr, col_idx = _csr(row_ptr, col_idx)
    M = row_ptr.size - 1
    priors = np.ascontiguousarray(priors, dtype=np.float64)
    N = priors.size
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    R = params.legs_after_first
    if gamma.shape != (R + 1, N):
        raise ValueError(f"gamma table must be [{R + 1}, {N}], got {gamma.shape}")
    sigma = np.ascontiguousarray(sigma, dtype=np.uint8)
    if sigma.ndim != 2 or sigma.shape[1] != M:
        raise ValueError("sigma must be uint8 [B, M]")
    B = sigma.shape[0]
    corr = np.zeros((B, N), dtype=np.uint8)
    legs = np.zeros(B, dtype=np.int32)
    conv = np.zeros(B, dtype=np.uint8)
    iters = np.zeros(B, dtype=np.int64)
    fin = np.zeros((B, N), dtype=np.float64) if want_marginals else None
    nt = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    clip = params.clip if params.clip > 0 else default_clip(precision)
    rc = _lib("relay", precision).oracle_relay_decode(
        M, N, _ptr(row_ptr), _ptr(col_idx), _ptr(priors), _ptr(gamma), R, params.iters_first,
        params.iters_later, params.max_total_iters, params.stop_after_solutions,
        params.warm_start_mode, clip, _ptr(sigma), B, _ptr(corr), _ptr(legs), _ptr(conv),
        _ptr(iters), _ptr(fin) if fin is not None else None, nt)
    if rc != 0:
        raise ValueError("oracle rejected its input")
    return RelayResult(corr, legs, conv, iters, fin)


def dmem_trace(row_ptr, col_idx, priors, gamma_row, sigma, T: int, clip: float = 0.0,
               precision: str = "f64", want_messages: bool = True, nthreads: int = 0):
    """T iterations of the first leg without early exit.

    Returns (Lambda [B, T, N], nu [B, T, E] or None, mu [B, T, E] or None), in
    float64; edges are in CSR order.
    """
    row_ptr, col_idx = _csr(row_ptr, col_idx)
    M = row_ptr.size - 1
    priors = np.ascontiguousarray(priors, dtype=np.float64)
    N = priors.size
    E = int(row_ptr[-1])
    gamma_row = np.ascontiguousarray(gamma_row, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.uint8)
    B = sigma.shape[0]
    Lam = np.zeros((B, T, N), dtype=np.float64)
    nu = np.zeros((B, T, E), dtype=np.float64) if want_messages else None
    mu = np.zeros((B, T, E), dtype=np.float64) if want_messages else None
    nt = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    clip = clip if clip > 0 else default_clip(precision)
    rc = _lib("relay", precision).oracle_dmem_trace(
        M, N, _ptr(row_ptr), _ptr(col_idx), _ptr(priors), _ptr(gamma_row), clip, _ptr(sigma), B,
        T, _ptr(Lam), _ptr(nu) if nu is not None else None,
        _ptr(mu) if mu is not None else None, nt)
    if rc != 0:
        raise ValueError("oracle rejected its input")
    return Lam, nu, mu
