"""Python binding of libqldpc.so (the C ABI in include/qldpc.h).

Argument marshalling only: every step of decoding runs in the library's CUDA
kernels.  The functions keep the C names; ``RelayDecoder`` wraps them for
PyTorch tensors (device memory and streams come from torch).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

QLDPC_OK = 0
QLDPC_ERR_INVALID_ARG = -1
QLDPC_ERR_CUDA = -2
QLDPC_ERR_OOM = -3
QLDPC_ERR_UNSUPPORTED = -4
QLDPC_MSG_FP32 = 0
QLDPC_MSG_FP16 = 1
QLDPC_KERNEL_AUTO = 0
QLDPC_KERNEL_BASELINE = 1
QLDPC_KERNEL_FUSED = 2

EXPORTED = ("qldpc_create", "qldpc_decode_batch", "qldpc_decode_batch_host",
            "qldpc_decode_batch_multi",
            "qldpc_decode_batch_host_static", "qldpc_trace_first_leg", "qldpc_get_info",
            "qldpc_destroy", "qldpc_status_string", "qldpc_last_error", "qldpc_soft_create",
            "qldpc_soft_workspace_bytes", "qldpc_soft_forward", "qldpc_soft_backward",
            "qldpc_soft_destroy", "qldpc_osd_create", "qldpc_osd_decode_batch",
            "qldpc_osd_destroy", "qldpc_cluster_create", "qldpc_cluster_decode_batch",
            "qldpc_cluster_destroy", "qldpc_grouped_workspace_bytes",
            "qldpc_decode_batch_grouped")
QLDPC_CLUSTER_SKIPPED = 0
QLDPC_CLUSTER_DECODED = 1
QLDPC_CLUSTER_TOO_LARGE = -1
QLDPC_CLUSTER_TOO_MANY = -2
QLDPC_CLUSTER_STALLED = -3
QLDPC_OSD_SKIPPED = 0
QLDPC_OSD_SOLVED = 1
QLDPC_OSD_TOO_MANY = -1
QLDPC_OSD_NO_SOLUTION = -2
QLDPC_REAL_FP32 = 0
QLDPC_REAL_FP64 = 1
QLDPC_STATIC_SCRATCH_BYTES = 8 * 1024 * 1024


class qldpc_relay_params(ctypes.Structure):
    _fields_ = [
        ("legs_after_first", ctypes.c_int32),
        ("iters_first", ctypes.c_int32),
        ("iters_later", ctypes.c_int32),
        ("max_total_iters", ctypes.c_int64),
        ("stop_after_solutions", ctypes.c_int32),
        ("warm_start_mode", ctypes.c_int32),
        ("msg_precision", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("llr_clip", ctypes.c_float),
        ("gamma_table", ctypes.c_void_p),
        ("tail_cut_iters", ctypes.c_int32),
    ]


class qldpc_osd_params(ctypes.Structure):
    _fields_ = [("bp_iters", ctypes.c_int32), ("llr_confident", ctypes.c_float),
                ("max_candidates", ctypes.c_int32)]


class qldpc_cluster_params(ctypes.Structure):
    _fields_ = [("bp_iters", ctypes.c_int32), ("llr_accept", ctypes.c_float),
                ("llr_erase", ctypes.c_float), ("max_clusters", ctypes.c_int32),
                ("max_cluster_faults", ctypes.c_int32)]


class qldpc_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "M", "N", "E", "max_check_degree", "max_fault_degree", "kernel", "msg_precision",
        "block_threads", "blocks_per_sm", "num_sms", "grid_blocks", "smem_bytes",
        "syndrome_words", "correction_words", "tail_cut_iters", "tail_block_threads",
        "tail_records")]


class QldpcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status}): {last_error()}")
        self.status = status


_LIB = None


def library_path() -> str:
    return _build.LIB


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libqldpc.so (built in-tree by __graft_entry__.build()); raise if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libqldpc.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.qldpc_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32, P, P, P,
                                 ctypes.POINTER(qldpc_relay_params), ctypes.c_int]
    lib.qldpc_decode_batch.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P]
    lib.qldpc_decode_batch_host.argtypes = [P, P, ctypes.c_int64, P, P, P, P]
    lib.qldpc_decode_batch_host_static.argtypes = [P, P, ctypes.c_int64, P, P, P, P]
    lib.qldpc_decode_batch_multi.argtypes = [P, ctypes.c_int32, P, P, ctypes.c_int32,
                                             ctypes.c_int64, P, ctypes.c_int32, P, P, P, P]
    lib.qldpc_grouped_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64]
    lib.qldpc_grouped_workspace_bytes.restype = ctypes.c_uint64
    lib.qldpc_decode_batch_grouped.argtypes = [P, ctypes.c_int32, P, P, ctypes.c_int32,
                                               ctypes.c_int64, P, ctypes.c_int32, P, P, P, P,
                                               ctypes.c_uint64, P]
    lib.qldpc_trace_first_leg.argtypes = [P, P, ctypes.c_int64, ctypes.c_int32, P, P, P, P]
    lib.qldpc_get_info.argtypes = [P, ctypes.POINTER(qldpc_info)]
    lib.qldpc_destroy.argtypes = [P]
    lib.qldpc_destroy.restype = None
    lib.qldpc_status_string.argtypes = [ctypes.c_int]
    lib.qldpc_status_string.restype = ctypes.c_char_p
    lib.qldpc_last_error.argtypes = []
    lib.qldpc_last_error.restype = ctypes.c_char_p
    lib.qldpc_osd_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32, P, P, P,
                                     ctypes.POINTER(qldpc_osd_params), ctypes.c_int]
    lib.qldpc_osd_decode_batch.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P]
    lib.qldpc_osd_destroy.argtypes = [P]
    lib.qldpc_osd_destroy.restype = None
    lib.qldpc_cluster_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32, P, P,
                                         P, ctypes.POINTER(qldpc_cluster_params), ctypes.c_int]
    lib.qldpc_cluster_decode_batch.argtypes = [P, P, ctypes.c_int64, P, P, P, P, P]
    lib.qldpc_cluster_destroy.argtypes = [P]
    lib.qldpc_cluster_destroy.restype = None
    lib.qldpc_soft_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32, P, P, P,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int]
    lib.qldpc_soft_workspace_bytes.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
    lib.qldpc_soft_forward.argtypes = [P, P, P, ctypes.c_int64, P, P, P, P, P, ctypes.c_uint64, P]
    lib.qldpc_soft_backward.argtypes = [P, P, P, ctypes.c_int64, P, P, P, P, P, P,
                                        ctypes.c_uint64, P]
    lib.qldpc_soft_destroy.argtypes = [P]
    lib.qldpc_soft_destroy.restype = None
    for name in ("qldpc_create", "qldpc_decode_batch", "qldpc_decode_batch_host",
                 "qldpc_decode_batch_multi",
                 "qldpc_decode_batch_host_static", "qldpc_trace_first_leg", "qldpc_get_info",
                 "qldpc_soft_create", "qldpc_soft_workspace_bytes", "qldpc_soft_forward",
                 "qldpc_soft_backward"):
        getattr(lib, name).restype = ctypes.c_int
    _LIB = lib
    return lib


def status_string(status: int) -> str:
    return load_library().qldpc_status_string(status).decode()


def last_error() -> str:
    return load_library().qldpc_last_error().decode()


def _check(status: int, what: str) -> None:
    if status != QLDPC_OK:
        raise QldpcError(status, what)


# ---- thin wrappers with the C names --------------------------------------------------

def qldpc_create(M, N, row_ptr, col_idx, priors, params: qldpc_relay_params, device=0):
    """Returns an opaque handle (ctypes.c_void_p).  Inputs are numpy host arrays."""
    lib = load_library()
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    _check(lib.qldpc_create(ctypes.byref(h), int(M), int(N), rp.ctypes.data, ci.ctypes.data,
                            pr.ctypes.data, ctypes.byref(params), int(device)), "qldpc_create")
    return h


def qldpc_decode_batch(h, syndromes_ptr, B, corrections_ptr, legs_ptr=None, conv_ptr=None,
                       iters_ptr=None, stream=None):
    _check(load_library().qldpc_decode_batch(h, syndromes_ptr, int(B), corrections_ptr,
                                             legs_ptr, conv_ptr, iters_ptr, stream),
           "qldpc_decode_batch")


def qldpc_decode_batch_host(h, syndromes_ptr, B, corrections_ptr, legs_ptr=None, conv_ptr=None,
                            iters_ptr=None):
    _check(load_library().qldpc_decode_batch_host(h, syndromes_ptr, int(B), corrections_ptr,
                                                  legs_ptr, conv_ptr, iters_ptr),
           "qldpc_decode_batch_host")


def qldpc_decode_batch_multi(handles, code_ptr, syn_ptr, syn_stride, B, cor_ptr, cor_stride,
                             legs_ptr=None, conv_ptr=None, iters_ptr=None, stream=None):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    _check(load_library().qldpc_decode_batch_multi(arr, len(handles), code_ptr, syn_ptr,
                                                   int(syn_stride), int(B), cor_ptr,
                                                   int(cor_stride), legs_ptr, conv_ptr, iters_ptr,
                                                   stream),
           "qldpc_decode_batch_multi")


def decode_mixed(decoders, code_of_shot, syndromes, stream=None):
    """Mixed batch through one persistent launch.

    decoders: list of RelayDecoder; code_of_shot: int32 CUDA tensor [B];
    syndromes: int64 CUDA tensor [B, stride] (each row starts with its code's
    ceil(M/64) words).  Returns (corrections [B, max ceil(N/64)], legs, converged, iters).
    """
    import torch
    B = syndromes.shape[0]
    cw = max(d.correction_words for d in decoders)
    dev = syndromes.device
    cor = torch.zeros((B, cw), dtype=torch.int64, device=dev)
    legs = torch.empty(B, dtype=torch.int32, device=dev)
    conv = torch.empty(B, dtype=torch.uint8, device=dev)
    iters = torch.empty(B, dtype=torch.int32, device=dev)
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    qldpc_decode_batch_multi([d.handle for d in decoders], ctypes.c_void_p(code_of_shot.data_ptr()),
                             ctypes.c_void_p(syndromes.data_ptr()), syndromes.shape[1], B,
                             ctypes.c_void_p(cor.data_ptr()), cw, ctypes.c_void_p(legs.data_ptr()),
                             ctypes.c_void_p(conv.data_ptr()), ctypes.c_void_p(iters.data_ptr()), st)
    return cor, legs, conv, iters


def qldpc_grouped_workspace_bytes(n_codes, B) -> int:
    return int(load_library().qldpc_grouped_workspace_bytes(int(n_codes), int(B)))


def qldpc_decode_batch_grouped(handles, code_ptr, syn_ptr, syn_stride, B, cor_ptr, cor_stride,
                               legs_ptr, conv_ptr, iters_ptr, ws_ptr, ws_bytes, stream=None):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    _check(load_library().qldpc_decode_batch_grouped(arr, len(handles), code_ptr, syn_ptr,
                                                     int(syn_stride), int(B), cor_ptr,
                                                     int(cor_stride), legs_ptr, conv_ptr,
                                                     iters_ptr, ws_ptr, int(ws_bytes), stream),
           "qldpc_decode_batch_grouped")


def decode_grouped(decoders, code_of_shot, syndromes, workspace=None, stream=None):
    """Mixed batch decoded per code with each decoder's own kernel shape (arguments and
    results as decode_mixed; `workspace` is a uint8 CUDA tensor of at least
    qldpc_grouped_workspace_bytes(len(decoders), B) bytes, allocated when None)."""
    import torch
    B = syndromes.shape[0]
    cw = max(d.correction_words for d in decoders)
    dev = syndromes.device
    need = qldpc_grouped_workspace_bytes(len(decoders), B)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    cor = torch.zeros((B, cw), dtype=torch.int64, device=dev)
    legs = torch.empty(B, dtype=torch.int32, device=dev)
    conv = torch.empty(B, dtype=torch.uint8, device=dev)
    iters = torch.empty(B, dtype=torch.int32, device=dev)
    st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    qldpc_decode_batch_grouped([d.handle for d in decoders],
                               ctypes.c_void_p(code_of_shot.data_ptr()),
                               ctypes.c_void_p(syndromes.data_ptr()), syndromes.shape[1], B,
                               ctypes.c_void_p(cor.data_ptr()), cw,
                               ctypes.c_void_p(legs.data_ptr()), ctypes.c_void_p(conv.data_ptr()),
                               ctypes.c_void_p(iters.data_ptr()),
                               ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), st)
    return cor, legs, conv, iters


def qldpc_decode_batch_host_static(h, syndromes_ptr, B, corrections_ptr, legs_ptr=None,
                                   conv_ptr=None, iters_ptr=None):
    """Host-buffer decode that allocates nothing (static device scratch; see qldpc.h)."""
    _check(load_library().qldpc_decode_batch_host_static(h, syndromes_ptr, int(B),
                                                         corrections_ptr, legs_ptr, conv_ptr,
                                                         iters_ptr),
           "qldpc_decode_batch_host_static")


def qldpc_trace_first_leg(h, syndromes_ptr, B, T, marg_ptr=None, nu_ptr=None, mu_ptr=None,
                          stream=None):
    _check(load_library().qldpc_trace_first_leg(h, syndromes_ptr, int(B), int(T), marg_ptr,
                                                nu_ptr, mu_ptr, stream),
           "qldpc_trace_first_leg")


def qldpc_get_info(h) -> qldpc_info:
    info = qldpc_info()
    _check(load_library().qldpc_get_info(h, ctypes.byref(info)), "qldpc_get_info")
    return info


def qldpc_destroy(h) -> None:
    if h is not None and h.value:
        load_library().qldpc_destroy(h)


# ---- torch convenience wrapper ------------------------------------------------------

@dataclass
class RelayConfig:
    """Relay parameters (paper App. A.3 defaults) plus kernel options."""
    legs_after_first: int = 300
    iters_first: int = 80
    iters_later: int = 60
    max_total_iters: int = 0
    stop_after_solutions: int = 1
    warm_start_mode: int = 0
    msg_precision: int = QLDPC_MSG_FP32
    kernel: int = QLDPC_KERNEL_AUTO
    block_threads: int = 0
    llr_clip: float = 0.0
    tail_cut_iters: int = 0   # 0: T_1 + 8 T_r; < 0: no tail continuation


class RelayDecoder:
    """A decoder for one decoding problem (H as CSR, priors, gamma table) on one GPU."""

    def __init__(self, row_ptr, col_idx, priors, gamma_table, config: RelayConfig | None = None,
                 device: int = 0):
        cfg = config or RelayConfig()
        self.config = cfg
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.M = row_ptr.size - 1
        self.N = int(np.asarray(priors).size)
        gam = np.ascontiguousarray(gamma_table, dtype=np.float32)
        if gam.shape != (cfg.legs_after_first + 1, self.N):
            raise ValueError(f"gamma table must be [{cfg.legs_after_first + 1}, {self.N}]")
        self._gamma = gam
        prm = qldpc_relay_params(cfg.legs_after_first, cfg.iters_first, cfg.iters_later,
                                 cfg.max_total_iters, cfg.stop_after_solutions,
                                 cfg.warm_start_mode, cfg.msg_precision, cfg.kernel,
                                 cfg.block_threads, cfg.llr_clip, gam.ctypes.data,
                                 cfg.tail_cut_iters)
        self.device = device
        self.handle = qldpc_create(self.M, self.N, row_ptr, col_idx, priors, prm, device)
        self.info = qldpc_get_info(self.handle)
        self.syndrome_words = self.info.syndrome_words
        self.correction_words = self.info.correction_words

    def close(self):
        if getattr(self, "handle", None) is not None:
            qldpc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream_ptr(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def outputs(self, B: int):
        import torch
        dev = torch.device("cuda", self.device)
        return (torch.empty((B, self.correction_words), dtype=torch.int64, device=dev),
                torch.empty(B, dtype=torch.int32, device=dev),
                torch.empty(B, dtype=torch.uint8, device=dev),
                torch.empty(B, dtype=torch.int32, device=dev))

    def decode(self, syndromes, out=None, stream=None):
        """syndromes: int64 CUDA tensor [B, ceil(M/64)] (bit-packed uint64 words).

        Returns (corrections int64 [B, ceil(N/64)], legs int32 [B], converged uint8 [B],
        iters int32 [B]), all on the device, enqueued on ``stream`` (default: torch's
        current stream).
        """
        if not syndromes.is_cuda or syndromes.dim() != 2 or \
                syndromes.shape[1] != self.syndrome_words or not syndromes.is_contiguous():
            raise ValueError("syndromes must be a contiguous CUDA tensor [B, ceil(M/64)]")
        B = syndromes.shape[0]
        cor, legs, conv, iters = out if out is not None else self.outputs(B)
        qldpc_decode_batch(self.handle, ctypes.c_void_p(syndromes.data_ptr()), B,
                           ctypes.c_void_p(cor.data_ptr()), ctypes.c_void_p(legs.data_ptr()),
                           ctypes.c_void_p(conv.data_ptr()), ctypes.c_void_p(iters.data_ptr()),
                           self._stream_ptr(stream))
        return cor, legs, conv, iters

    def decode_host(self, syndromes: np.ndarray, out=None):
        """Host-buffer path: numpy uint64 [B, ceil(M/64)] in, numpy arrays out (synchronous)."""
        syn = np.ascontiguousarray(syndromes, dtype=np.uint64)
        if syn.ndim != 2 or syn.shape[1] != self.syndrome_words:
            raise ValueError("syndromes must be uint64 [B, ceil(M/64)]")
        B = syn.shape[0]
        if out is None:
            out = (np.empty((B, self.correction_words), dtype=np.uint64),
                   np.empty(B, dtype=np.int32), np.empty(B, dtype=np.uint8),
                   np.empty(B, dtype=np.int32))
        cor, legs, conv, iters = out
        qldpc_decode_batch_host(self.handle, ctypes.c_void_p(syn.ctypes.data), B,
                                ctypes.c_void_p(cor.ctypes.data), ctypes.c_void_p(legs.ctypes.data),
                                ctypes.c_void_p(conv.ctypes.data),
                                ctypes.c_void_p(iters.ctypes.data))
        return out

    def trace_first_leg(self, syndromes, T: int, messages: bool = True, stream=None):
        """Lambda(t), nu(t), mu(t) for t = 1..T of the first leg (no early exit)."""
        import torch
        B = syndromes.shape[0]
        dev = syndromes.device
        marg = torch.empty((T, B, self.N), dtype=torch.float32, device=dev)
        nu = torch.empty((T, B, self.info.E), dtype=torch.float32, device=dev) if messages else None
        mu = torch.empty((T, B, self.info.E), dtype=torch.float32, device=dev) if messages else None
        qldpc_trace_first_leg(self.handle, ctypes.c_void_p(syndromes.data_ptr()), B, T,
                              ctypes.c_void_p(marg.data_ptr()),
                              ctypes.c_void_p(nu.data_ptr()) if messages else None,
                              ctypes.c_void_p(mu.data_ptr()) if messages else None,
                              self._stream_ptr(stream))
        return marg, nu, mu


# ---- soft DMem-BP (differentiable leg) ----------------------------------------------

def qldpc_soft_create(M, N, row_ptr, col_idx, priors, iterations, checkpoint_every, real_type,
                      device=0):
    lib = load_library()
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    _check(lib.qldpc_soft_create(ctypes.byref(h), int(M), int(N), rp.ctypes.data, ci.ctypes.data,
                                 pr.ctypes.data, int(iterations), int(checkpoint_every),
                                 int(real_type), int(device)), "qldpc_soft_create")
    return h


def qldpc_soft_workspace_bytes(h, B) -> int:
    n = ctypes.c_uint64()
    _check(load_library().qldpc_soft_workspace_bytes(h, int(B), ctypes.byref(n)),
           "qldpc_soft_workspace_bytes")
    return int(n.value)


def qldpc_soft_forward(h, syn_ptr, faults_ptr, B, gamma_ptr, alpha_ptr, loss_ptr, marg_ptr,
                       ws_ptr, ws_bytes, stream=None):
    _check(load_library().qldpc_soft_forward(h, syn_ptr, faults_ptr, int(B), gamma_ptr, alpha_ptr,
                                             loss_ptr, marg_ptr, ws_ptr, int(ws_bytes), stream),
           "qldpc_soft_forward")


def qldpc_soft_backward(h, syn_ptr, faults_ptr, B, gamma_ptr, alpha_ptr, loss_grad_ptr,
                        grad_gamma_ptr, grad_alpha_ptr, ws_ptr, ws_bytes, stream=None):
    _check(load_library().qldpc_soft_backward(h, syn_ptr, faults_ptr, int(B), gamma_ptr,
                                              alpha_ptr, loss_grad_ptr, grad_gamma_ptr,
                                              grad_alpha_ptr, ws_ptr, int(ws_bytes), stream),
           "qldpc_soft_backward")


def qldpc_soft_destroy(h) -> None:
    if h is not None and h.value:
        load_library().qldpc_soft_destroy(h)


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class SoftDMem:
    """Unrolled soft DMem-BP leg on one GPU (see include/qldpc.h for the equations).

    dtype: torch.float32 or torch.float64 (every real tensor passed in must match).
    """

    def __init__(self, row_ptr, col_idx, priors, iterations: int = 25,
                 checkpoint_every: int = 5, dtype=None, device: int = 0):
        import torch
        self.dtype = dtype or torch.float32
        real = QLDPC_REAL_FP64 if self.dtype == torch.float64 else QLDPC_REAL_FP32
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.M, self.N = row_ptr.size - 1, int(np.asarray(priors).size)
        self.T, self.K, self.device = iterations, checkpoint_every, device
        self.handle = qldpc_soft_create(self.M, self.N, row_ptr, col_idx, priors, iterations,
                                        checkpoint_every, real, device)

    def close(self):
        if getattr(self, "handle", None) is not None:
            qldpc_soft_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, B: int):
        import torch
        n = qldpc_soft_workspace_bytes(self.handle, B)
        return torch.empty(n, dtype=torch.uint8, device=torch.device("cuda", self.device))

    def forward(self, syndromes, faults, gamma, alpha, workspace=None, marginals=False,
                stream=None):
        """Returns (loss [1], Lambda(T) [B, N] or None, workspace)."""
        import torch
        B = syndromes.shape[0]
        ws = workspace if workspace is not None else self.workspace(B)
        loss = torch.empty(1, dtype=self.dtype, device=gamma.device)
        marg = torch.empty((B, self.N), dtype=self.dtype, device=gamma.device) if marginals else None
        st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        qldpc_soft_forward(self.handle, _vp(syndromes), _vp(faults), B, _vp(gamma), _vp(alpha),
                           _vp(loss), _vp(marg), _vp(ws), ws.numel(), st)
        return loss, marg, ws

    def backward(self, syndromes, faults, gamma, alpha, workspace, loss_grad=None, stream=None):
        """Returns (grad_gamma [N], grad_alpha [T]); needs the forward's workspace."""
        import torch
        B = syndromes.shape[0]
        gg = torch.empty(self.N, dtype=self.dtype, device=gamma.device)
        ga = torch.empty(self.T, dtype=self.dtype, device=gamma.device)
        st = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        qldpc_soft_backward(self.handle, _vp(syndromes), _vp(faults), B, _vp(gamma), _vp(alpha),
                            _vp(loss_grad), _vp(gg), _vp(ga), _vp(workspace), workspace.numel(),
                            st)
        return gg, ga


def soft_dmem_loss(soft: SoftDMem, syndromes, faults, gamma, alpha):
    """Loss of the unrolled soft DMem-BP leg, differentiable in gamma and alpha.

    syndromes / faults: int64 CUDA tensors of bit-packed words [B, ceil(M/64)] and
    [B, ceil(N/64)]; gamma [N], alpha [T]: CUDA tensors of soft.dtype.
    """
    return _SoftDMemLoss.apply(gamma, alpha, soft, syndromes, faults)


def _autograd_function():
    import torch

    class SoftDMemLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, gamma, alpha, soft, syndromes, faults):
            gamma = gamma.contiguous()
            alpha = alpha.contiguous()
            loss, _, ws = soft.forward(syndromes, faults, gamma, alpha)
            ctx.soft = soft
            ctx.save_for_backward(gamma, alpha, syndromes, faults, ws)
            return loss.reshape(())

        @staticmethod
        def backward(ctx, grad_loss):
            gamma, alpha, syndromes, faults, ws = ctx.saved_tensors
            up = grad_loss.reshape(1).to(gamma.dtype).contiguous()
            gg, ga = ctx.soft.backward(syndromes, faults, gamma, alpha, ws, loss_grad=up)
            return gg, ga, None, None, None

    return SoftDMemLoss


class _Lazy:
    def __init__(self):
        self.fn = None

    def apply(self, *args):
        if self.fn is None:
            self.fn = _autograd_function()
        return self.fn.apply(*args)


_SoftDMemLoss = _Lazy()


# ---- filtered-OSD post-processor -----------------------------------------------------

def qldpc_osd_create(M, N, row_ptr, col_idx, priors, params: qldpc_osd_params, device=0):
    lib = load_library()
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    _check(lib.qldpc_osd_create(ctypes.byref(h), int(M), int(N), rp.ctypes.data, ci.ctypes.data,
                                pr.ctypes.data, ctypes.byref(params), int(device)),
           "qldpc_osd_create")
    return h


def qldpc_osd_decode_batch(h, syn_ptr, B, skip_ptr, cor_ptr, status_ptr, ncand_ptr=None,
                           stream=None):
    _check(load_library().qldpc_osd_decode_batch(h, syn_ptr, int(B), skip_ptr, cor_ptr,
                                                 status_ptr, ncand_ptr, stream),
           "qldpc_osd_decode_batch")


def qldpc_osd_destroy(h) -> None:
    if h is not None and h.value:
        load_library().qldpc_osd_destroy(h)


class FilteredOSD:
    """Filtered-OSD post-processor for one decoding problem on one GPU (paper Sec. 5)."""

    def __init__(self, row_ptr, col_idx, priors, bp_iters: int = 25,
                 llr_confident: float = 8.0, max_candidates: int = 500, device: int = 0):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.M = row_ptr.size - 1
        self.N = int(np.asarray(priors).size)
        self.params = qldpc_osd_params(bp_iters, llr_confident, max_candidates)
        self.device = device
        self.handle = qldpc_osd_create(self.M, self.N, row_ptr, col_idx, priors, self.params,
                                       device)
        self.syndrome_words = (self.M + 63) // 64
        self.correction_words = (self.N + 63) // 64

    def close(self):
        if getattr(self, "handle", None) is not None:
            qldpc_osd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, syndromes, corrections, skip=None, status=None, n_candidates=None,
               stream=None):
        """Post-process the shots with skip == 0 (all shots when skip is None).

        syndromes int64 [B, ceil(M/64)] and corrections int64 [B, ceil(N/64)] (updated in
        place for solved shots) are CUDA tensors; returns (status int32 [B],
        n_candidates int32 [B]).
        """
        import torch
        B = syndromes.shape[0]
        if syndromes.shape != (B, self.syndrome_words) or not syndromes.is_contiguous():
            raise ValueError("syndromes must be a contiguous CUDA tensor [B, ceil(M/64)]")
        if corrections.shape != (B, self.correction_words) or not corrections.is_contiguous():
            raise ValueError("corrections must be a contiguous CUDA tensor [B, ceil(N/64)]")
        dev = syndromes.device
        status = status if status is not None else torch.empty(B, dtype=torch.int32, device=dev)
        ncand = n_candidates if n_candidates is not None else torch.empty(B, dtype=torch.int32,
                                                                          device=dev)
        s = stream if stream is not None else torch.cuda.current_stream()
        qldpc_osd_decode_batch(self.handle, ctypes.c_void_p(syndromes.data_ptr()), B,
                               _vp(skip) if skip is not None else None,
                               ctypes.c_void_p(corrections.data_ptr()),
                               ctypes.c_void_p(status.data_ptr()),
                               ctypes.c_void_p(ncand.data_ptr()), ctypes.c_void_p(s.cuda_stream))
        return status, ncand


def first_leg_then_osd(first_leg: "RelayDecoder", osd: FilteredOSD, syndromes, stream=None):
    """The post-processed decoder of the paper's comparison (Sec. 7.1): the first Relay
    leg (a RelayDecoder with legs_after_first = 0) on every shot, filtered-OSD on the
    shots it leaves unconverged.  Returns (corrections, status, n_candidates, converged)
    with status QLDPC_OSD_SKIPPED where the first leg converged."""
    cor, _, conv, _ = first_leg.decode(syndromes, stream=stream)
    status, ncand = osd.decode(syndromes, cor, skip=conv, stream=stream)
    return cor, status, ncand, conv


# ---- cluster decoder ------------------------------------------------------------------

def qldpc_cluster_create(M, N, row_ptr, col_idx, priors, params: qldpc_cluster_params,
                         device=0):
    lib = load_library()
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    pr = np.ascontiguousarray(priors, dtype=np.float64)
    _check(lib.qldpc_cluster_create(ctypes.byref(h), int(M), int(N), rp.ctypes.data,
                                    ci.ctypes.data, pr.ctypes.data, ctypes.byref(params),
                                    int(device)), "qldpc_cluster_create")
    return h


def qldpc_cluster_decode_batch(h, syn_ptr, B, skip_ptr, cor_ptr, status_ptr, steps_ptr=None,
                               stream=None):
    _check(load_library().qldpc_cluster_decode_batch(h, syn_ptr, int(B), skip_ptr, cor_ptr,
                                                     status_ptr, steps_ptr, stream),
           "qldpc_cluster_decode_batch")


def qldpc_cluster_destroy(h) -> None:
    if h is not None and h.value:
        load_library().qldpc_cluster_destroy(h)


class ClusterDecoder:
    """BP + generalized union-find cluster decoder for one decoding problem on one GPU
    (paper Sec. 2.5 and Sec. 6)."""

    def __init__(self, row_ptr, col_idx, priors, bp_iters: int = 25, llr_accept: float = -0.5,
                 llr_erase: float = 4.5, max_clusters: int = 128,
                 max_cluster_faults: int = 512, device: int = 0):
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.M = row_ptr.size - 1
        self.N = int(np.asarray(priors).size)
        self.params = qldpc_cluster_params(bp_iters, llr_accept, llr_erase, max_clusters,
                                           max_cluster_faults)
        self.device = device
        self.handle = qldpc_cluster_create(self.M, self.N, row_ptr, col_idx, priors,
                                           self.params, device)
        self.syndrome_words = (self.M + 63) // 64
        self.correction_words = (self.N + 63) // 64

    def close(self):
        if getattr(self, "handle", None) is not None:
            qldpc_cluster_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def decode(self, syndromes, corrections, skip=None, status=None, steps=None, stream=None):
        """Decode the shots with skip == 0 (all when skip is None).  syndromes int64
        [B, ceil(M/64)] and corrections int64 [B, ceil(N/64)] (updated in place for decoded
        shots) are CUDA tensors; returns (status int32 [B], steps int32 [B])."""
        import torch
        B = syndromes.shape[0]
        if syndromes.shape != (B, self.syndrome_words) or not syndromes.is_contiguous():
            raise ValueError("syndromes must be a contiguous CUDA tensor [B, ceil(M/64)]")
        if corrections.shape != (B, self.correction_words) or not corrections.is_contiguous():
            raise ValueError("corrections must be a contiguous CUDA tensor [B, ceil(N/64)]")
        dev = syndromes.device
        status = status if status is not None else torch.empty(B, dtype=torch.int32, device=dev)
        steps = steps if steps is not None else torch.empty(B, dtype=torch.int32, device=dev)
        s = stream if stream is not None else torch.cuda.current_stream()
        qldpc_cluster_decode_batch(self.handle, ctypes.c_void_p(syndromes.data_ptr()), B,
                                   _vp(skip) if skip is not None else None,
                                   ctypes.c_void_p(corrections.data_ptr()),
                                   ctypes.c_void_p(status.data_ptr()),
                                   ctypes.c_void_p(steps.data_ptr()),
                                   ctypes.c_void_p(s.cuda_stream))
        return status, steps


def first_leg_then_cluster(first_leg: "RelayDecoder", cluster: ClusterDecoder, syndromes,
                           stream=None):
    """First Relay leg on every shot, BP + cluster decoding on the shots it leaves
    unconverged (paper Sec. 7.1).  Returns (corrections, status, steps, converged)."""
    cor, _, conv, _ = first_leg.decode(syndromes, stream=stream)
    status, steps = cluster.decode(syndromes, cor, skip=conv, stream=stream)
    return cor, status, steps, conv
