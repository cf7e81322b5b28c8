"""ctypes front end of the soft DMem-BP oracle (TEST INFRASTRUCTURE ONLY).

One unrolled leg of DMem-BP with the sum-product check rule, per-iteration scale
alpha_t and per-fault memory strengths gamma_j; BCE loss of the final marginals
against the true faults; gradient by a plain reverse pass over the stored
trajectory (see soft_dmem_oracle.c for the equations).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_P = ctypes.c_void_p
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.lib_path("soft", "f64")
        if not os.path.exists(path):
            _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_soft_dmem.restype = ctypes.c_int
        lib.oracle_soft_dmem.argtypes = [
            ctypes.c_int32, ctypes.c_int32, _P, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_double,
            _P, _P, ctypes.c_int64, _P, _P, _P, _P, ctypes.c_int32]
        _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def soft_dmem(row_ptr, col_idx, priors, gamma, alpha, sigma, F, eps: float = 1e-15,
              grad: bool = True, marginals: bool = False, nthreads: int = 0):
    """Returns (loss, grad_gamma [N] or None, grad_alpha [T] or None, Lambda(T) [B,N] or None)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    priors = np.ascontiguousarray(priors, dtype=np.float64)
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.uint8)
    F = np.ascontiguousarray(F, dtype=np.uint8)
    M, N, T, B = row_ptr.size - 1, priors.size, alpha.size, sigma.shape[0]
    if gamma.shape != (N,) or sigma.shape != (B, M) or F.shape != (B, N):
        raise ValueError("shape mismatch")
    loss = np.zeros(1)
    gg = np.zeros(N) if grad else None
    ga = np.zeros(T) if grad else None
    marg = np.zeros((B, N)) if marginals else None
    nt = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    rc = _lib().oracle_soft_dmem(M, N, _p(row_ptr), _p(col_idx), _p(priors), T, _p(gamma),
                                 _p(alpha), eps, _p(sigma), _p(F), B, _p(loss), _p(gg), _p(ga),
                                 _p(marg), nt)
    if rc != 0:
        raise ValueError("oracle rejected its input")
    return float(loss[0]), gg, ga, marg
